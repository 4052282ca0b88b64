// Host driver of the TT-UTV sweep and the C ABI declared in include/ttutv.h.
//
// One sweep step factors the current unfolding C (row-major m x n, a free
// view of the previous carry).  The basis side is the column side for URV
// (right-to-left, Alg. 3) and the row side for ULV (left-to-right, Alg. 1/2);
// N_b is its size and N_o the other side's.
//   exact path  (N_b <= l_full): G = Gram of the basis side (FP64), small
//               factor of G -> Z_1, r; carry = C Z_1 (URV) or Z_1^T C (ULV).
//   sketch path (N_b  > l_full): Y = C^T Omega (URV) / C Omega (ULV) with a
//               Rademacher Omega (identity when l >= N_o), W = CholeskyQR2(Y),
//               B = C W (URV) / C^T W (ULV), small factor of B^T B -> Z_1, r;
//               core from W Z_1, carry from B Z_1.  l grows (x2) when the rank
//               needs more than l - p columns or the tolerance is missed.
// The rank of each step is read back through pinned host memory (the only
// synchronization of the step); everything else stays on the stream.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <string>
#include <type_traits>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "internal.h"
#include "ttutv.h"

namespace {

thread_local std::string g_err;

tt_status fail(tt_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

tt_status cuda_fail(cudaError_t e, const char* what) {
  return fail(TT_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define TT_CK(expr, what)                         \
  do {                                            \
    cudaError_t e_ = (expr);                      \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

// Host-time accounting of a sweep (printed with TTUTV_DEBUG=2): wall time,
// time blocked in the per-step synchronizations, time inside the caller's
// allocator, and the number of allocator calls.
double host_us() {
  return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now().time_since_epoch())
      .count();
}
struct HostProf {
  double alloc_us = 0.0, sync_us = 0.0;
  int nalloc = 0;
};
thread_local HostProf g_hprof;

struct Alloc {
  tt_alloc_fn al;
  tt_free_fn fr;
  void* ctx;
  cudaStream_t st;
  void* get(size_t bytes) {
    const double t0 = host_us();
    bytes = ((bytes ? bytes : 1) + 255) & ~(size_t)255;
    void* p = nullptr;
    if (al) {
      p = al(bytes, (void*)st, ctx);
    } else if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
    }
    g_hprof.alloc_us += host_us() - t0;
    ++g_hprof.nalloc;
    return p;
  }
  void put(void* p) {
    if (!p) return;
    const double t0 = host_us();
    if (fr)
      fr(p, (void*)st, ctx);
    else
      cudaFreeAsync(p, st);
    g_hprof.alloc_us += host_us() - t0;
    ++g_hprof.nalloc;
  }
};

// Device buffer released through the caller's allocator at scope exit.
struct Buf {
  Alloc* a;
  void* p = nullptr;
  explicit Buf(Alloc* a_) : a(a_) {}
  Buf(const Buf&) = delete;
  ~Buf() { reset(); }
  void reset() {
    if (p) a->put(p);
    p = nullptr;
  }
  bool get(size_t bytes) {
    reset();
    p = a->get(bytes);
    return p != nullptr;
  }
  void* release() {
    void* q = p;
    p = nullptr;
    return q;
  }
  template <typename T>
  T* as() const {
    return (T*)p;
  }
};

#define TT_ALLOC(buf, bytes)                                                         \
  do {                                                                               \
    if (!(buf).get(bytes)) return fail(TT_ENOMEM, "allocator returned NULL");        \
  } while (0)

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// One scratch block per sweep, carved step by step: every scratch buffer of
// a step comes out of it, so a sweep makes a few allocator calls instead of
// one per buffer (each is a round trip into the caller's allocator).  A step
// reserves the total of its carve-outs first; the block only grows (with 25%
// headroom, released stream-ordered) when a step needs more than it holds.
struct Scratch {
  Alloc* a;
  void* p = nullptr;
  size_t cap = 0, off = 0;
  explicit Scratch(Alloc* a_) : a(a_) {}
  Scratch(const Scratch&) = delete;
  ~Scratch() {
    if (p) a->put(p);
  }
  bool reserve(size_t total) {
    off = 0;
    if (total <= cap) return true;
    if (p) a->put(p);
    cap = total + total / 4;
    p = a->get(cap);
    if (!p) cap = 0;
    return p != nullptr;
  }
  void* take(size_t bytes) {
    bytes = align256(bytes ? bytes : 1);
    if (!p || off + bytes > cap) return nullptr;
    void* q = (char*)p + off;
    off += bytes;
    return q;
  }
};

// A buffer carved from the step's Scratch (released with it).
struct Piece {
  void* p = nullptr;
  template <typename T>
  T* as() const {
    return (T*)p;
  }
};

#define TT_RESERVE(scr, bytes)                                                      \
  do {                                                                              \
    if (!(scr).reserve(bytes)) return fail(TT_ENOMEM, "allocator returned NULL");   \
  } while (0)
#define TT_TAKE(piece, bytes)                                                       \
  do {                                                                              \
    (piece).p = scr.take(bytes);                                                    \
    if (!(piece).p) return fail(TT_ENOMEM, "step scratch larger than reserved");    \
  } while (0)

ttk::StepInfo* pinned_info() {
  thread_local ttk::StepInfo* h = nullptr;
  thread_local ttk::StepInfo fallback;
  if (!h) {
    if (cudaMallocHost((void**)&h, sizeof(ttk::StepInfo)) != cudaSuccess) {
      cudaGetLastError();
      h = &fallback;
    }
  }
  return h;
}

// Pinned copy of the device error word of the tensor-core kernels.
int* pinned_err() {
  thread_local int* h = nullptr;
  thread_local int fallback = 0;
  if (!h) {
    if (cudaMallocHost((void**)&h, sizeof(int)) != cudaSuccess) {
      cudaGetLastError();
      h = &fallback;
    }
  }
  return h;
}

int64_t roundup(int64_t x, int64_t m) { return ((x + m - 1) / m) * m; }

// TTUTV_DEBUG=1 prints one line per sweep step to stderr.
bool host_prof() {
  static const bool on = [] {
    const char* v = getenv("TTUTV_DEBUG");
    return v && v[0] == '2';
  }();
  return on;
}

bool debug_trace() {
  static const bool on = [] {
    const char* v = getenv("TTUTV_DEBUG");
    return v && v[0] == '1';
  }();
  return on;
}

// Test hook: TTUTV_JACOBI_SWEEPS=k caps the TT-SVD Jacobi iteration at k
// sweeps (default 60), so that a test can reach TT_ENOCONV without a fault.
int jacobi_sweeps() {
  static const int k = [] {
    const char* v = getenv("TTUTV_JACOBI_SWEEPS");
    const int x = v ? atoi(v) : 0;
    return x > 0 && x < 60 ? x : 0;
  }();
  return k;
}

// Sketch width l: r + p for a fixed rank, else roundup16(max(2 r_prev,
// r_prev + p, 32)); never more than either side nor the small-factor limit.
int64_t sketch_size(int64_t nb, int64_t no, int64_t r_prev, int64_t p, int64_t rfix) {
  int64_t l = (rfix >= 1) ? rfix + p : roundup(std::max<int64_t>(std::max<int64_t>(2 * r_prev, r_prev + p), 32), 16);
  l = std::min<int64_t>(l, std::min<int64_t>(nb, no));
  return std::min<int64_t>(l, ttk::kMaxSmall);
}

// CUDA-event timing of the sweep's phases (only when opts.phase_ms is set).
// Events come from a per-thread pool that is created once and reused, so a
// timed sweep adds only event records to its stream.  Every phase is also an
// NVTX range ("step s: phase"), free unless a profiler is attached.
struct PhaseTimer {
  bool nvtx_open = false;
  ~PhaseTimer() {
    if (nvtx_open) nvtxRangePop();
  }
  double* out = nullptr;
  cudaStream_t st = nullptr;
  struct Rec {
    int step, phase;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  int open = -1;
  static std::vector<cudaEvent_t>& pool() {
    thread_local std::vector<cudaEvent_t> p;
    return p;
  }
  size_t used = 0;  // events of the pool taken by this sweep
  cudaEvent_t take() {
    auto& p = pool();
    if (used == p.size()) {
      cudaEvent_t e = nullptr;
      if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
      }
      p.push_back(e);
    }
    return p[used++];
  }
  void begin(int step, int phase) {
    static const char* const names[TT_NPHASES] = {"gram", "small", "carry", "core",
                                                  "sketch", "orth", "project", "other"};
    char label[48];
    snprintf(label, sizeof label, "step %d: %s", step, names[phase & 7]);
    if (nvtx_open) nvtxRangePop();
    nvtxRangePushA(label);
    nvtx_open = true;
    if (!out) return;
    Rec r{step, phase, take(), take()};
    if (!r.a || !r.b) return;
    cudaEventRecord(r.a, st);
    recs.push_back(r);
    open = (int)recs.size() - 1;
  }
  void end() {
    if (nvtx_open) {
      nvtxRangePop();
      nvtx_open = false;
    }
    if (!out || open < 0) return;
    cudaEventRecord(recs[open].b, st);
    open = -1;
  }
  // after a stream synchronization; the pool's events are free again
  void collect() {
    for (auto& r : recs) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess && out)
        out[r.step * TT_NPHASES + r.phase] += ms;
      cudaGetLastError();
    }
    recs.clear();
    used = 0;
  }
};

// Product routing.  With TT_P_MIXED, FP32 products run on the tensor cores
// (tc_gemm: TF32 operands, split hi + lo where the product is part of the
// kept factor) when their operands are eligible; Gram matrices that must
// resolve errors below FP32 rounding (accurate) and everything else run on
// the SIMT kernels (gemm<W>).
struct MM {
  bool tc;
  int* err;
  cudaStream_t st;
};

template <typename W>
size_t mm_ws(const MM& mm, int64_t M, int64_t N, int64_t K, bool sym_or_out64) {
  size_t b = ttk::gemm_ws_bytes<W>(M, N, K, sym_or_out64);
  if constexpr (std::is_same<W, float>::value) {
    if (mm.tc)
      b = std::max(b, ttk::tc_gemm_ws_bytes(M, N, K, sym_or_out64, sym_or_out64, true, true));
  }
  return b;
}

template <typename W>
cudaError_t mm_run(const MM& mm, ttk::Mat<W> A, ttk::Mat<W> B, int64_t M, int64_t N, int64_t K,
                   W* out, int64_t ldo, double* out64, bool sym, double* sumsq, void* ws,
                   bool accurate, bool a_split, bool b_split, bool round_out) {
  if constexpr (std::is_same<W, float>::value) {
    if (mm.tc && !accurate) {
      ttk::TcOpts o;
      o.a_split = a_split;
      o.b_split = b_split;
      o.round_out = round_out;
      o.err = mm.err;
      cudaError_t e = ttk::tc_gemm(A, B, M, N, K, out, ldo, out64, sym, sumsq, ws, mm.st, o);
      if (e != cudaErrorNotSupported) return e;
      cudaGetLastError();
    }
  }
  return ttk::gemm<W>(A, B, M, N, K, out, ldo, out64, sym, sumsq, ws, mm.st, accurate);
}

struct SweepCfg {
  bool urv;   // basis on the column side, right-to-left
  bool svd;   // Jacobi small factor (TT-SVD)
  bool l11 = false;  // appendix Alg. 4 keeping L_11 alone (TT-ULV right-to-left)
};

// True for host memory (pageable or pinned), false for device memory.
bool host_pointer(const void* p) {
  cudaPointerAttributes pa;
  if (cudaPointerGetAttributes(&pa, p) != cudaSuccess) {
    cudaGetLastError();
    return true;
  }
  return pa.type == cudaMemoryTypeHost || pa.type == cudaMemoryTypeUnregistered;
}

// Rows of C per slab of the direct residual: about 64 MiB of residual at a
// time, a multiple of 4 rows (slab offsets stay 16-byte aligned for TMA).
int64_t residual_slab(int64_t rows, int64_t cols, size_t elem) {
  int64_t per = (int64_t)((64ull << 20) / ((size_t)std::max<int64_t>(cols, 1) * elem));
  per = std::max<int64_t>(4, per & ~(int64_t)3);
  return std::max<int64_t>(1, std::min<int64_t>(rows, per));
}

template <typename W>
tt_status run_sweep(const void* A_in, int32_t dtype_in, int d, const int64_t* dims, double eps,
                    const int64_t* fixed, SweepCfg cfg, const tt_opts& o, Alloc& al,
                    tt_result* out, const tt_shard* sh = nullptr) {
  constexpr bool W64 = std::is_same<W, double>::value;
  cudaStream_t st = al.st;
  const int64_t p_over = o.oversample;
  const int64_t l_full = o.l_full;

  // equal weights: sum w_k^2 = 1 (errors orthogonal, Thm 3.1), or for Alg. 4
  // keeping L_11 alone, whose errors add in norm, sum w_k = 1 (its Proposition)
  std::vector<double> w(d - 1, cfg.l11 ? 1.0 / (double)(d - 1) : 1.0 / sqrt((double)(d - 1)));
  if (o.weights)
    for (int i = 0; i < d - 1; ++i) w[i] = o.weights[i];

  // Partition over ranks (tt_utv_sharded): every rank holds the slab
  // rank * slab .. of the partitioned mode (mode 1 for the right-to-left URV
  // sweep, whose unfoldings keep it as their slowest row index; mode d for
  // the left-to-right ULV sweep, their fastest column index).  dl are the
  // local mode sizes; the unfoldings stay partitioned (`active`) until a step
  // needs a whole unfolding (an identity sketch gathers it).
  bool active = sh && sh->nranks > 1;
  const int pm = cfg.urv ? 0 : d - 1;
  int64_t dl[TT_MAXD];
  for (int k = 0; k < d; ++k) dl[k] = dims[k];
  const int64_t slab = active ? dims[pm] / sh->nranks : dims[pm];
  if (active) dl[pm] = slab;
  auto reduce = [&](double* buf, int64_t count) -> tt_status {
    if (!active) return TT_OK;
    const int32_t r = sh->allreduce(buf, count, (void*)st, sh->ctx);
    return r == 0 ? TT_OK : fail(r > 0 && r <= TT_EUNSUPPORTED ? (tt_status)r : TT_ECUDA,
                                 "the all-reduce callback failed");
  };
  auto gather = [&](const void* send, void* recv, int64_t bytes) -> tt_status {
    const int32_t r = sh->allgather(send, recv, bytes, (void*)st, sh->ctx);
    return r == 0 ? TT_OK : fail(r > 0 && r <= TT_EUNSUPPORTED ? (tt_status)r : TT_ECUDA,
                                 "the all-gather callback failed");
  };
#define TT_RED(buf, count)                        \
  do {                                            \
    const tt_status rs_ = reduce((buf), (count)); \
    if (rs_ != TT_OK) return rs_;                 \
  } while (0)

  int64_t total = 1;
  for (int k = 0; k < d; ++k) total *= dl[k];

  // Input in the working precision, on the device.
  const bool host_in = host_pointer(A_in);
  const bool in64 = dtype_in == TT_F64;
  const size_t in_el = in64 ? 8 : 4;
  Buf staged(&al), conv(&al);
  const void* src = A_in;
  if (host_in) {
    TT_ALLOC(staged, total * in_el);
    TT_CK(cudaMemcpyAsync(staged.p, A_in, total * in_el, cudaMemcpyHostToDevice, st), "copy input");
    src = staged.p;
  }
  const W* A = (const W*)src;
  if (in64 != W64) {
    TT_ALLOC(conv, total * sizeof(W));
    TT_CK(ttk::cast_copy(src, in64, conv.p, W64, total, st), "widen/narrow input");
    A = conv.as<W>();
    staged.reset();
  }

  // sweep-long device records: scalars, per-step carry norms, the error
  // word and the small factor's StepInfo, in one block
  const size_t scal_bytes = align256(sizeof(double) * (4 + 2 * TT_MAXD));
  Buf scal(&al);
  TT_ALLOC(scal, scal_bytes + sizeof(ttk::StepInfo));
  double* d_scal = scal.as<double>();
  double* d_x2first = d_scal;            // ||A||^2 when the first step is sketched
  double* d_carry2 = d_scal + 4;         // per step: ||carry||^2 (sum of squares of stored values)
  double* d_tdirect = d_scal + 4 + TT_MAXD;  // per step: a directly summed tail (identity sketch)
  std::vector<char> has_direct(d, 0);
  int* d_err = (int*)(d_scal + 1);       // set by a tensor-core kernel whose bounded wait ran out
  TT_CK(cudaMemsetAsync(d_scal, 0, sizeof(double) * (4 + 2 * TT_MAXD), st), "memset");
  int* herr = pinned_err();
  const bool mixed = !W64 && o.precision == TT_P_MIXED;
  const MM mm_all{mixed, d_err, st};
  Piece dinfo;
  dinfo.p = (char*)scal.p + scal_bytes;
  ttk::StepInfo* hinfo = pinned_info();
  Scratch scr(&al);

  memset(out, 0, sizeof(*out));
  out->d = d;
  out->dtype = W64 ? TT_F64 : TT_F32;
  out->orth = cfg.urv ? 0 : 1;
  for (int k = 0; k < d; ++k) out->dims[k] = dims[k];
  out->ranks[0] = out->ranks[d] = 1;

  std::vector<void*> cores(d, nullptr);
  struct CoreGuard {
    std::vector<void*>& c;
    Alloc& a;
    bool ok = false;
    ~CoreGuard() {
      if (!ok)
        for (void* p : c) a.put(p);
    }
  } guard{cores, al};

  PhaseTimer tm;
  tm.out = o.phase_ms;
  tm.st = st;
  std::vector<double> x2s(d, 0.0);
  std::vector<double> ftail(d, -1.0);
  const W* C = A;
  Buf cbuf(&al);
  double normA2 = -1.0;
  int64_t r_carry = 1, r_prev = 0;

  for (int s = 0; s < d - 1; ++s) {
    const int k = cfg.urv ? d - s : s + 1;  // core being separated (1-based)
    int64_t m, n, m_g, n_g;  // local and global unfolding sizes
    {
      const int64_t* cd = active ? dl : dims;
      if (cfg.urv) {
        m = m_g = 1;
        for (int t = 0; t < k - 1; ++t) {
          m *= cd[t];
          m_g *= dims[t];
        }
        n = n_g = dims[k - 1] * r_carry;
      } else {
        m = m_g = r_carry * dims[k - 1];
        n = n_g = 1;
        for (int t = k; t < d; ++t) {
          n *= cd[t];
          n_g *= dims[t];
        }
      }
    }
    const int u = cfg.urv ? k - 1 : k;  // unfolding number 1..d-1
    // nb: the basis side (never partitioned); no: the other side's local
    // size, no_g its size over all ranks (it decides the sketch)
    const int64_t nb = cfg.urv ? n : m, no_g = cfg.urv ? m_g : n_g;
    int64_t no = cfg.urv ? m : n;
    const double dscale = fixed ? 0.0 : (w[u - 1] * eps) * (w[u - 1] * eps);
    const int64_t rfix = fixed ? fixed[u - 1] : -1;
    // A tolerance within a few FP32 ulps of ||C||^2 (eps_k^2 below 2e-7 of
    // ||A||^2, about 3.4 u) cannot be resolved from FP32-summed products: the
    // range miss mu^2 = ||C||^2 - ||C P_W||^2 of a sketched step comes out
    // with an error of several 1e-9 of ||C||^2 whatever the sketch width, and
    // at tighter tolerances FP32 accumulation (or the tensor cores' drift)
    // buries the kept directions themselves in the sketch, the range basis,
    // the projection, the carry and the core.  Every product of such a step
    // uses compensated sums of exact products on the SIMT path, and the
    // projection B = C W is kept in FP64 for its Gram: rounding B to FP32
    // alone perturbs ||B||^2 by ~u ||C||^2 / sqrt(rows).
    const bool precise = !W64 && !fixed && dscale < 2e-7;
    const int64_t rcap = std::min<int64_t>(std::min<int64_t>(nb, no_g), ttk::kMaxSmall);
    const bool exact = nb <= l_full;
    const bool first = (s == 0);

    // A tolerance below ~n u_fp32 of ||C||^2 cannot be resolved from an
    // FP32-accumulated Gram or an FP32 factorization: such steps form the
    // Gram with compensated sums of exact products, and factor it in FP64.
    auto tight = [&](int64_t nsz) {
      return !fixed && !(dscale >= 2.0 * (double)nsz * 5.9604644775390625e-08);
    };
    // double-float small factors (FP32 data only): FP64-grade in every use
    const bool small_df = !W64 && o.small_precision == TT_SMALL_DF;
    auto choose_small64 = [&](int64_t nsz) {
      if (o.small_precision == TT_SMALL_FP64 || small_df) return true;
      if (o.small_precision == TT_SMALL_FP32) return false;
      if (W64) return true;
      return tight(nsz);
    };

    ttk::SmallParams prm;
    memset(&prm, 0, sizeof(prm));
    prm.mode = cfg.svd ? ttk::SM_JACOBI
                       : (o.inner == TT_INNER_USVP   ? ttk::SM_USVP
                          : o.inner == TT_INNER_LURV ? ttk::SM_LURV
                                                     : ttk::SM_QLP);
    prm.usvp_iters = o.usvp_iters;
    prm.l11 = cfg.l11 ? 1 : 0;
    prm.jacobi_sweeps = jacobi_sweeps();
    prm.r_fixed = (int)rfix;
    prm.r_cap = (int)rcap;
    prm.delta2_scale = dscale;
    prm.delta2 = (normA2 >= 0.0) ? dscale * normA2 : 0.0;

    Buf carry(&al), core(&al), ws_extra(&al);
    Buf cfull(&al);  // the whole unfolding, gathered for an identity sketch
    Piece zb, ws, ws2, gb, omega, yb, s1b, w1b, wb, bb, gy, gwb, tb;
    size_t ws_bytes = 0;  // size of ws (reused by the carry and core products)
    int64_t r = 1, l = 0;
    bool small64 = false;
    bool acc_gram = false;  // the factored Gram was formed with compensated sums
    const W* Zp = nullptr;
    const W* Wfin = nullptr;  // final sketch basis (sketch path)
    int64_t ldz = 0;

    // A tight step's range finding (Grams, sketch, projection) runs on the
    // SIMT path: its tail estimates must be unbiased below FP32 rounding,
    // which the tensor cores' accumulation is not.
    MM mm = mm_all;
    if (exact) {
      mm.tc = mm_all.tc && !tight(nb);
      // the carry product's scratch is bounded by its widest rank
      const int64_t rmax = rcap;
      ws_bytes = std::max(mm_ws<W>(mm, nb, nb, no, true), ttk::small_ws_bytes((int)nb, true));
      ws_bytes = std::max(ws_bytes, cfg.urv ? mm_ws<W>(mm_all, m, rmax, n, false)
                                            : mm_ws<W>(mm_all, rmax, n, m, false));
      TT_RESERVE(scr, align256((size_t)nb * nb * sizeof(double)) + align256((size_t)nb * nb * sizeof(W)) +
                          align256(ws_bytes) + (cfg.l11 ? align256((size_t)nb * nb * sizeof(W)) : 0));
      TT_TAKE(gb, (size_t)nb * nb * sizeof(double));
      TT_TAKE(zb, (size_t)nb * nb * sizeof(W));
      if (cfg.l11) TT_TAKE(tb, (size_t)nb * nb * sizeof(W));
      TT_TAKE(ws, ws_bytes);
      const bool acc = !W64 && tight(nb);
      acc_gram = acc;
      tm.begin(s, TT_PH_GRAM);
      if (cfg.urv)
        TT_CK(mm_run<W>(mm, {C, n, false}, {C, n, true}, n, n, m, nullptr, 0, gb.as<double>(), true,
                        nullptr, ws.p, acc, false, false, false), "Gram C^T C");
      else
        TT_CK(mm_run<W>(mm, {C, n, true}, {C, n, false}, m, m, n, nullptr, 0, gb.as<double>(), true,
                        nullptr, ws.p, acc, false, false, false), "Gram C C^T");
      TT_RED(gb.as<double>(), nb * nb);
      tm.end();
      small64 = choose_small64(nb);
      prm.n = (int)nb;
      if (first) {
        prm.normA2_dev = d_scal;  // any non-null pointer: the value is this Gram's trace
        prm.normA2_is_trace = 1;
      }
      prm.x2_dev = nullptr;
      prm.piv_tol = small64 ? (small_df ? 1e-13 : 1e-15) : 1e-6;
      prm.df_math = small_df ? 1 : 0;
      ldz = nb;
      prm.Tl = tb.p;
      tm.begin(s, TT_PH_SMALL);
      TT_CK(ttk::small_factor(gb.as<double>(), prm, small64, zb.p, W64, (int)ldz, ws.p,
                              dinfo.as<ttk::StepInfo>(), st), "small factor");
      tm.end();
      TT_CK(cudaMemcpyAsync(hinfo, dinfo.p, sizeof(ttk::StepInfo), cudaMemcpyDeviceToHost, st), "info");
      TT_CK(cudaMemcpyAsync(herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, st), "error word");
      {
        const double t0 = host_us();
        TT_CK(cudaStreamSynchronize(st), "step sync");
        g_hprof.sync_us += host_us() - t0;
      }
      tm.collect();
      if (*herr) return fail(TT_ETIMEOUT, "a bounded wait in a tensor-core kernel ran out");
      if (hinfo->status & 1) return fail(TT_ENONFINITE, "input holds NaN or Inf");
      if (hinfo->status & 2) return fail(TT_ENOCONV, "Jacobi eigen-solver did not converge");
      r = hinfo->r;
      Zp = zb.as<W>();
    } else {
      l = sketch_size(nb, no_g, r_prev, p_over, rfix);
      const double* x2_dev = first ? d_x2first : (d_carry2 + (s - 1));
      if (first) {
        TT_RESERVE(scr, ttk::sumsq_ws_bytes(total));
        Piece sw;
        TT_TAKE(sw, ttk::sumsq_ws_bytes(total));
        TT_CK(ttk::sumsq(C, W64, m * n, d_x2first, sw.p, st), "sum of squares");
        TT_RED(d_x2first, 1);
        prm.normA2_dev = d_x2first;
        prm.normA2_is_trace = 0;
      }
      while (true) {
        const bool identity = l >= no_g;
        if (identity && active) {
          // Omega = I needs the whole unfolding: gather it; this step and the
          // rest of the sweep then run on every rank alike
          const int64_t lb = m * n;
          Buf gb_all(&al);
          TT_ALLOC(cfull, (size_t)m_g * n_g * sizeof(W));
          if (cfg.urv) {
            const tt_status sg = gather(C, cfull.p, lb * (int64_t)sizeof(W));
            if (sg != TT_OK) return sg;
          } else {
            TT_ALLOC(gb_all, (size_t)lb * sh->nranks * sizeof(W));
            const tt_status sg = gather(C, gb_all.p, lb * (int64_t)sizeof(W));
            if (sg != TT_OK) return sg;
            TT_CK(ttk::unshard_cols(gb_all.p, cfull.p, W64, sh->nranks, m, n / dl[d - 1], dl[d - 1], st),
                  "interleave gathered columns");
          }
          C = cfull.as<W>();
          m = m_g;
          n = n_g;
          no = no_g;
          active = false;
        }
        small64 = choose_small64(l);
        mm.tc = mm_all.tc && !tight(l);
        const bool powered = o.power_iters > 0 && !identity;
        const bool whiten_l = !W64 && small64;
        {
          // this width's carve-outs (the previous width's are dead)
          size_t wsz = 0;
          wsz = std::max(wsz, mm_ws<W>(mm, nb, l, no, false));
          wsz = std::max(wsz, mm_ws<W>(mm, l, l, nb, true));
          wsz = std::max(wsz, mm_ws<W>(mm, nb, l, l, false));
          wsz = std::max(wsz, mm_ws<W>(mm, no, l, nb, false));
          wsz = std::max(wsz, mm_ws<W>(mm, l, l, no, true));
          const int64_t rmax = std::min<int64_t>(rcap, l);
          wsz = std::max(wsz, cfg.urv ? mm_ws<W>(mm_all, m, rmax, l, false)
                                      : mm_ws<W>(mm_all, rmax, n, l, false));
          wsz = std::max(wsz, cfg.urv ? mm_ws<W>(mm_all, rmax, n, l, false)
                                      : mm_ws<W>(mm_all, m, rmax, l, false));
          if (precise) wsz = std::max(wsz, mm_ws<double>(mm, l, l, no, true));
          ws_bytes = wsz;
          const size_t nl = align256((size_t)nb * l * sizeof(W)), ol = align256((size_t)no * l * sizeof(W));
          const size_t ll8 = align256((size_t)l * l * sizeof(double)), llw = align256((size_t)l * l * sizeof(W));
          size_t tot = (identity ? 0 : ol) + nl + align256(wsz) + align256(ttk::small_ws_bytes((int)l, true)) +
                       ll8 + llw + 2 * nl + ol + (whiten_l ? ll8 : 0) + llw + (cfg.l11 ? llw : 0);
          if (powered) tot += ol;
          if (precise) tot += align256((size_t)no * l * sizeof(double));  // B in FP64
          if (active) {
            // a slab's partial sketch is formed in FP64 and summed over ranks
            wsz = std::max(wsz, mm_ws<W>(mm, nb, l, no, true));
            ws_bytes = wsz;
            tot += align256(wsz) + align256((size_t)nb * l * sizeof(double));
          }
          TT_RESERVE(scr, tot);
        }
        if (!identity) TT_TAKE(omega, (size_t)no * l * sizeof(W));
        tm.begin(s, TT_PH_SKETCH);
        if (!identity) {
          // a slab draws the sketch rows of its own rows (URV: a contiguous
          // block of rows; ULV: the columns of its slab of mode d, strided)
          const int64_t blk = !active ? 0 : (cfg.urv ? no : dl[d - 1]);
          const int64_t stride = cfg.urv ? 0 : dims[d - 1];
          const int64_t off = !active ? 0 : (int64_t)sh->rank * (cfg.urv ? no : dl[d - 1]);
          TT_CK(ttk::fill_sketch(omega.p, W64, no, l, o.seed, (uint32_t)k, false, st, blk, stride, off),
                "sketch matrix");
        }
        TT_TAKE(yb, (size_t)nb * l * sizeof(W));
        TT_TAKE(ws, ws_bytes);
        TT_TAKE(ws2, ttk::small_ws_bytes((int)l, true));
        Piece y64;  // a slab's partial sketch in FP64
        if (active) TT_TAKE(y64, (size_t)nb * l * sizeof(double));
        // Y = sum over ranks of the slabs' partial sketches (FP64), rounded once
        auto sum_sketch = [&]() -> tt_status {
          TT_RED(y64.as<double>(), nb * l);
          TT_CK(ttk::cast_copy(y64.p, true, yb.p, W64, nb * l, st), "sketch to working precision");
          return TT_OK;
        };
        // Omega = I (l = N_o): Y is C^T / C itself, copied exactly.  On the
        // tensor cores C is split into two TF32 terms (Omega = +-1 is exact):
        // TF32 rounding noise in Y would enter every sketch column at ~2^-12
        // of its norm, outside the row space of C, and tilt the basis.
        if (identity && cfg.urv)
          TT_CK(ttk::copy2d(C, n, true, yb.p, l, nb, l, W64, st), "sketch C^T");
        else if (identity)
          TT_CK(ttk::copy2d(C, n, false, yb.p, l, nb, l, W64, st), "sketch C");
        else if (cfg.urv)
          TT_CK(mm_run<W>(mm, {C, n, false}, {omega.as<W>(), l, true}, n, l, m, active ? nullptr : yb.as<W>(),
                          l, active ? y64.as<double>() : nullptr, false, nullptr, ws.p, precise, true, false,
                          false), "sketch C^T Omega");
        else
          TT_CK(mm_run<W>(mm, {C, n, true}, {omega.as<W>(), l, true}, m, l, n, active ? nullptr : yb.as<W>(),
                          l, active ? y64.as<double>() : nullptr, false, nullptr, ws.p, precise, true, false,
                          false), "sketch C Omega");
        if (active && !identity) {
          const tt_status sr = sum_sketch();
          if (sr != TT_OK) return sr;
        }
        tm.end();

        // Shifted Cholesky-QR3: a shifted pass that cannot break down, then two
        // plain passes; span(out[:, :j]) = span(src[:, :j]) for every j, the
        // basis Householder QR gives up to column signs.
        TT_TAKE(gy, (size_t)l * l * sizeof(double));
        TT_TAKE(s1b, (size_t)l * l * sizeof(W));
        TT_TAKE(w1b, (size_t)nb * l * sizeof(W));
        TT_TAKE(wb, (size_t)nb * l * sizeof(W));
        ttk::SmallParams po;
        memset(&po, 0, sizeof(po));
        po.n = (int)l;
        po.mode = ttk::SM_ORTH;
        po.r_fixed = -1;
        po.r_cap = (int)l;
        // With a tight tolerance the sketch may carry directions near the
        // FP32 floor; W_1 is then too ill-conditioned for an FP32-summed
        // Gram to stay positive definite, so those Grams use compensated sums
        // of exact products and the Cholesky runs in FP64.
        const bool orth_df = !W64 && o.orth_precision == TT_SMALL_DF;
        po.df_math = orth_df ? 1 : 0;
        const bool orth64 = o.orth_precision == TT_SMALL_FP64 || orth_df ||
                            (o.orth_precision == TT_SMALL_AUTO && (small64 || W64));
        // unit roundoff of the Cholesky's arithmetic (double-float: ~2^-48)
        const double u_c = orth_df ? 3.552713678800501e-15
                                   : orth64 ? 1.1102230246251565e-16 : 5.9604644775390625e-08;
        // three passes src -> d0 -> d1 -> d0; returns d0
        auto orth3 = [&](const W* src, W* d0, W* d1) -> tt_status {
          W* dst[3] = {d0, d1, d0};
          for (int pass = 0; pass < 3; ++pass) {
            // the smallest shift that keeps the first Cholesky positive definite
            // (a few l u of the Gram's scale): a larger one squashes the sketch's
            // weak directions, and the later passes then amplify rounding in them
            po.shift_rel = pass == 0 ? 4.0 * (double)l * u_c : 0.0;
            po.piv_tol = pass == 0 ? 0.0 : 64.0 * (double)l * u_c * u_c;
            TT_CK(mm_run<W>(mm, {src, l, false}, {src, l, true}, l, l, nb, nullptr, 0,
                            gy.as<double>(), true, nullptr, ws.p, !W64 && small64, true, true, false),
                  "Gram of sketch");
            TT_CK(ttk::small_factor(gy.as<double>(), po, orth64, s1b.p, W64, (int)l, ws2.p,
                                    dinfo.as<ttk::StepInfo>(), st), "orthonormalize");
            TT_CK(mm_run<W>(mm, {src, l, true}, {s1b.as<W>(), l, true}, nb, l, l, dst[pass], l,
                            nullptr, false, nullptr, ws.p, precise, true, true, false), "apply R^-1");
            src = dst[pass];
          }
          return TT_OK;
        };
        // q power (subspace) iterations: Y <- X^T X Q with Q the orthonormal
        // basis of the previous Y (Cholesky-QR3, nested spans as above); X = C
        // (URV) or C^T (ULV).  The same products as the sketch and the projection.
        if (powered) {
          Piece pb;
          TT_TAKE(pb, (size_t)no * l * sizeof(W));
          tm.begin(s, TT_PH_SKETCH);
          for (int it = 0; it < o.power_iters; ++it) {
            const tt_status so = orth3(yb.as<W>(), w1b.as<W>(), wb.as<W>());
            if (so != TT_OK) return so;
            const W* Q = w1b.as<W>();
            if (cfg.urv) {
              TT_CK(mm_run<W>(mm, {C, n, true}, {Q, l, true}, m, l, n, pb.as<W>(), l, nullptr,
                              false, nullptr, ws.p, false, true, true, false), "power iteration: C Q");
              TT_CK(mm_run<W>(mm, {C, n, false}, {pb.as<W>(), l, true}, n, l, m, active ? nullptr : yb.as<W>(),
                              l, active ? y64.as<double>() : nullptr, false, nullptr, ws.p, false, true,
                              true, false), "power iteration: C^T P");
            } else {
              TT_CK(mm_run<W>(mm, {C, n, false}, {Q, l, true}, n, l, m, pb.as<W>(), l, nullptr,
                              false, nullptr, ws.p, false, true, true, false), "power iteration: C^T Q");
              TT_CK(mm_run<W>(mm, {C, n, true}, {pb.as<W>(), l, true}, m, l, n, active ? nullptr : yb.as<W>(),
                              l, active ? y64.as<double>() : nullptr, false, nullptr, ws.p, false, true,
                              true, false), "power iteration: C P");
            }
            if (active) {
              const tt_status sr = sum_sketch();
              if (sr != TT_OK) return sr;
            }
          }
          tm.end();
        }
        tm.begin(s, TT_PH_ORTH);
        {
          const tt_status so = orth3(yb.as<W>(), w1b.as<W>(), wb.as<W>());
          if (so != TT_OK) return so;
        }
        const W* src_pass = w1b.as<W>();
        tm.end();
        const W* Wm = src_pass;
        Wfin = Wm;
        TT_TAKE(bb, (size_t)no * l * sizeof(W));
        Piece bb64;  // a precise step's projection in FP64, for its Gram
        if (precise) TT_TAKE(bb64, (size_t)no * l * sizeof(double));
        double* b64 = precise ? bb64.as<double>() : nullptr;
        acc_gram = !W64 && tight(l);
        tm.begin(s, TT_PH_PROJECT);
        if (cfg.urv)
          TT_CK(mm_run<W>(mm, {C, n, true}, {Wm, l, true}, m, l, n, bb.as<W>(), l, b64, false,
                          nullptr, ws.p, precise, true, true, false), "project C W");
        else
          TT_CK(mm_run<W>(mm, {C, n, false}, {Wm, l, true}, n, l, m, bb.as<W>(), l, b64, false,
                          nullptr, ws.p, precise, true, true, false), "project C^T W");
        if (precise)
          TT_CK(mm_run<double>(mm, {b64, l, false}, {b64, l, true}, l, l, no, nullptr, 0,
                               gy.as<double>(), true, nullptr, ws.p, false, false, false, false),
                "Gram B^T B (FP64)");
        else
          TT_CK(mm_run<W>(mm, {bb.as<W>(), l, false}, {bb.as<W>(), l, true}, l, l, no, nullptr, 0,
                          gy.as<double>(), true, nullptr, ws.p, acc_gram, true, true, false),
                "Gram B^T B");
        TT_RED(gy.as<double>(), l * l);
        // FP32 W is orthonormal only to ~1e-7, which biases ||X W||^2 and so
        // the range miss mu^2; with a tight tolerance the small factor
        // whitens by W^T W (compensated sums of exact products).
        const bool whiten = whiten_l;
        if (whiten) {
          TT_TAKE(gwb, (size_t)l * l * sizeof(double));
          TT_CK(mm_run<W>(mm, {Wm, l, false}, {Wm, l, true}, l, l, nb, nullptr, 0, gwb.as<double>(),
                          true, nullptr, ws.p, true, false, false, false), "Gram W^T W");
        }
        prm.Gw = whiten ? gwb.as<double>() : nullptr;
        tm.end();
        prm.n = (int)l;
        prm.r_cap = (int)std::min<int64_t>(rcap, l);
        prm.x2_dev = x2_dev;
        prm.range_exact = identity ? 1 : 0;
        prm.piv_tol = small64 ? (small_df ? 1e-13 : 1e-15) : 1e-6;
        prm.df_math = small_df ? 1 : 0;
        TT_TAKE(zb, (size_t)l * l * sizeof(W));
        if (cfg.l11) TT_TAKE(tb, (size_t)l * l * sizeof(W));
        prm.Tl = tb.p;
        ldz = l;
        tm.begin(s, TT_PH_SMALL);
        TT_CK(ttk::small_factor(gy.as<double>(), prm, small64, zb.p, W64, (int)ldz, ws2.p,
                                dinfo.as<ttk::StepInfo>(), st), "small factor");
        tm.end();
        TT_CK(cudaMemcpyAsync(hinfo, dinfo.p, sizeof(ttk::StepInfo), cudaMemcpyDeviceToHost, st), "info");
        TT_CK(cudaMemcpyAsync(herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, st), "error word");
        {
          const double t0 = host_us();
          TT_CK(cudaStreamSynchronize(st), "step sync");
          g_hprof.sync_us += host_us() - t0;
        }
        tm.collect();
        if (*herr) return fail(TT_ETIMEOUT, "a bounded wait in a tensor-core kernel ran out");
        if (hinfo->status & 1) return fail(TT_ENONFINITE, "input holds NaN or Inf");
        if (hinfo->status & 2) return fail(TT_ENOCONV, "Jacobi eigen-solver did not converge");
        r = hinfo->r;
        const double d2 = hinfo->delta2;
        const int64_t lmax = std::min<int64_t>(std::min<int64_t>(nb, no), ttk::kMaxSmall);
        if (debug_trace())
          fprintf(stderr, "[ttutv]   sketch attempt k=%d l=%lld r=%d mu2=%.3e s1=%.3e tail=%.3e delta2=%.3e x2=%.9e trace=%.9e\n",
                  k, (long long)l, hinfo->r, hinfo->mu2, hinfo->s1, hinfo->tail, d2, hinfo->x2, hinfo->trace);
        if (!fixed && (r > l - p_over || hinfo->tail > d2)) {
          if (l < lmax) {
            l = std::min<int64_t>(2 * l, lmax);
            continue;
          }
          if (hinfo->tail > d2)
            return fail(TT_EUNSUPPORTED, "prescribed accuracy needs a rank above the 256-column sketch");
        }
        break;
      }
      Zp = zb.as<W>();
    }

    if (first) normA2 = hinfo->normA2;
    x2s[s] = hinfo->x2;
    // A tight step's tail from the small factor (compensated Gram, FP64
    // factorization) resolves errors far below FP32 rounding; the difference
    // ||C||^2 - ||carry||^2 is limited by the carry's own rounding (and by the
    // tensor cores' accumulation drift, ~1e-6 of ||C||^2) and is used otherwise.
    ftail[s] = (acc_gram && small64) ? hinfo->tail : -1.0;
    if (debug_trace())
      fprintf(stderr,
              "[ttutv] step k=%d %s m=%lld n=%lld l=%lld small=%s r=%d k1=%d nsteps=%d x2=%.6e "
              "trace=%.6e mu2=%.3e s1=%.3e delta2=%.3e tail=%.3e status=%d\n",
              k, exact ? "exact" : "sketch", (long long)m, (long long)n, (long long)l,
              small64 ? "fp64" : "fp32", hinfo->r, hinfo->k1, hinfo->nsteps, hinfo->x2,
              hinfo->trace, hinfo->mu2, hinfo->s1, hinfo->delta2, hinfo->tail, hinfo->status);
    out->delta_sq[u - 1] = fixed ? 0.0 : hinfo->delta2;
    out->sketch_l[u - 1] = exact ? 0 : (int32_t)l;
    out->small_fp64[u - 1] = small64 ? 1 : 0;

    // carry and core.  A tight step's carry and core may use the tensor
    // cores again: neither enters this step's tail, and the next step forms
    // its tail from the carry as stored (its sum of squares and its Gram), so
    // a ~2^-22 relative error in the carry only adds ~2^-44 of its squared
    // norm to that tail.
    mm = mm_all;
    if (precise) mm.tc = false;
    // The next step's ||C||^2 is this carry's sum of squares.  The tensor-core
    // epilogue sums each row's squares in FP32 (~u/sqrt(rows) relative); after
    // a tight step the carry's squares are summed again exactly (FP64).
    const bool sq_pass = mm.tc && acc_gram;
    double* carry_sq = sq_pass ? nullptr : d_carry2 + s;
    const int64_t crow = cfg.urv ? m : r, ccol = cfg.urv ? r : n;
    TT_ALLOC(carry, (size_t)crow * ccol * sizeof(W));
    const int64_t corerows = cfg.urv ? r : m, corecols = cfg.urv ? n : r;
    TT_ALLOC(core, (size_t)corerows * corecols * sizeof(W));
    {
      size_t wsz = 0;
      if (exact) {
        wsz = cfg.urv ? mm_ws<W>(mm, m, r, n, false) : mm_ws<W>(mm, r, n, m, false);
      } else {
        wsz = std::max(cfg.urv ? mm_ws<W>(mm, m, r, l, false) : mm_ws<W>(mm, r, n, l, false),
                       cfg.urv ? mm_ws<W>(mm, r, n, l, false) : mm_ws<W>(mm, m, r, l, false));
        if (l >= no_g && r < l)  // the identity sketch's residual product
          wsz = std::max(wsz, cfg.urv ? mm_ws<W>(mm, m, l, r, false) : mm_ws<W>(mm, n, l, r, false));
      }
      if (o.direct_tails)  // the residual product of one slab of rows
        wsz = std::max(wsz, mm_ws<W>(mm, residual_slab(m, n, sizeof(W)), n, r, false));
      if (sq_pass) wsz = std::max(wsz, ttk::sumsq_ws_bytes(crow * ccol));
      if (wsz > ws_bytes) {
        TT_ALLOC(ws_extra, wsz);
        ws.p = ws_extra.p;
      }
    }
    if (exact) {
      tm.begin(s, TT_PH_CARRY);
      if (cfg.urv)
        TT_CK(mm_run<W>(mm, {C, n, true}, {cfg.l11 ? tb.as<W>() : Zp, ldz, true}, m, r, n,
                        carry.as<W>(), r, nullptr, false, carry_sq, ws.p, precise, true, true, false),
              cfg.l11 ? "carry C T (U_1 L_11)" : "carry C Z1");
      else
        TT_CK(mm_run<W>(mm, {Zp, ldz, false}, {C, n, true}, r, n, m, carry.as<W>(), n, nullptr, false,
                        carry_sq, ws.p, precise, true, true, false), "carry Z1^T C");
      tm.end();
      tm.begin(s, TT_PH_CORE);
      if (cfg.urv)
        TT_CK(ttk::copy2d(Zp, ldz, true, core.p, n, r, n, W64, st), "core Z1^T");
      else
        TT_CK(ttk::copy2d(Zp, ldz, false, core.p, r, m, r, W64, st), "core Z1");
      tm.end();
    } else {
      const W* Bm = bb.as<W>();
      const W* Wm = Wfin;
      tm.begin(s, TT_PH_CARRY);
      if (cfg.urv)
        TT_CK(mm_run<W>(mm, {Bm, l, true}, {cfg.l11 ? tb.as<W>() : Zp, ldz, true}, m, r, l,
                        carry.as<W>(), r, nullptr, false, carry_sq, ws.p, precise, true, true, false),
              cfg.l11 ? "carry B T (U_1 L_11)" : "carry B Z1");
      else
        TT_CK(mm_run<W>(mm, {Zp, ldz, false}, {Bm, l, false}, r, n, l, carry.as<W>(), n, nullptr, false,
                        carry_sq, ws.p, precise, true, true, false), "carry (B Z1)^T");
      tm.end();
      // Omega = I: W spans the whole row space (mu^2 = 0), so the step's
      // error is ||B - B Z1 Z1^T||^2, summed directly from that residual
      // instead of as ||C||^2 - ||carry||^2, where the products' rounding
      // (~1e-6 of ||C||^2 on the tensor cores) swamps a small tail
      if (!exact && l >= no_g && r < l && !cfg.l11 && ftail[s] < 0.0) {
        const int64_t nbl = (cfg.urv ? m : n) * l;
        const size_t pbytes = align256(ttk::diff_sumsq_parts_bytes());
        Buf trail(&al);
        TT_ALLOC(trail, align256((size_t)nbl * sizeof(W)) + pbytes + 2 * sizeof(double));
        W* Pm = trail.as<W>();
        double* part = (double*)((char*)trail.p + align256((size_t)nbl * sizeof(W)));
        double* pair = (double*)((char*)part + pbytes);
        // P = carry Z1^T in B's layout (URV: m x l row-major; ULV: B^T, n x l)
        if (cfg.urv)
          TT_CK(mm_run<W>(mm, {carry.as<W>(), r, true}, {Zp, ldz, false}, m, l, r, Pm, l, nullptr,
                          false, nullptr, ws.p, precise, true, true, false),
                "carry Z1^T");
        else
          TT_CK(mm_run<W>(mm, {carry.as<W>(), n, false}, {Zp, ldz, false}, n, l, r, Pm, l, nullptr,
                          false, nullptr, ws.p, precise, true, true, false),
                "carry^T Z1^T");
        TT_CK(ttk::diff_sumsq(Bm, Pm, W64, nbl, part, true, st), "residual of the identity sketch");
        TT_CK(ttk::sum_pairs(part, pair, st), "residual of the identity sketch");
        TT_CK(cudaMemcpyAsync(d_tdirect + s, pair, sizeof(double), cudaMemcpyDeviceToDevice, st),
              "residual of the identity sketch");
        has_direct[s] = 1;
      }
      tm.begin(s, TT_PH_CORE);
      if (cfg.urv)
        TT_CK(mm_run<W>(mm, {Zp, ldz, false}, {Wm, l, false}, r, n, l, core.as<W>(), n, nullptr, false,
                        nullptr, ws.p, precise, true, true, false), "core (W Z1)^T");
      else
        TT_CK(mm_run<W>(mm, {Wm, l, true}, {Zp, ldz, true}, m, r, l, core.as<W>(), r, nullptr, false,
                        nullptr, ws.p, precise, true, true, false), "core W Z1");
      tm.end();
    }
    // Opt-in (tt_opts.direct_tails): the step's error ||E_k||^2 summed
    // directly from its residual, URV E = C - carry Z1^T, ULV E = C - Z1
    // carry (the core is Z1^T, resp. Z1), formed slab by slab of C's rows
    // and summed in FP64 -- instead of ||C||^2 - ||carry||^2, whose
    // tensor-core rounding (~1e-6 of ||C||^2) is the size of a sketched
    // step's range miss.  Exact and sketched steps alike (identity sketches
    // and tight steps already report direct errors).  Ranks and cores are
    // unchanged.  On a partitioned sweep every rank sums its slab and the
    // sums are all-reduced.
    if (o.direct_tails && !has_direct[s] && !cfg.l11 && ftail[s] < 0.0) {
      const int64_t slab = residual_slab(m, n, sizeof(W));
      const size_t pbytes = align256(ttk::diff_sumsq_parts_bytes());
      Buf trail(&al);
      TT_ALLOC(trail, align256((size_t)slab * n * sizeof(W)) + pbytes + 2 * sizeof(double));
      W* Pm = trail.as<W>();
      double* part = (double*)((char*)trail.p + align256((size_t)slab * n * sizeof(W)));
      double* pair = (double*)((char*)part + pbytes);
      for (int64_t a = 0; a < m; a += slab) {
        const int64_t h = std::min(slab, m - a);
        if (cfg.urv)
          TT_CK(mm_run<W>(mm, {carry.as<W>() + a * r, r, true}, {core.as<W>(), n, true}, h, n, r, Pm,
                          n, nullptr, false, nullptr, ws.p, precise, true, true, false),
                "step residual: carry Z1^T");
        else
          TT_CK(mm_run<W>(mm, {core.as<W>() + a * r, r, true}, {carry.as<W>(), n, true}, h, n, r, Pm,
                          n, nullptr, false, nullptr, ws.p, precise, true, true, false),
                "step residual: Z1 carry");
        TT_CK(ttk::diff_sumsq(C + a * n, Pm, W64, h * n, part, a == 0, st), "step residual");
      }
      TT_CK(ttk::sum_pairs(part, pair, st), "step residual");
      TT_CK(cudaMemcpyAsync(d_tdirect + s, pair, sizeof(double), cudaMemcpyDeviceToDevice, st),
            "step residual");
      TT_RED(d_tdirect + s, 1);
      has_direct[s] = 1;
    }
    if (sq_pass)
      TT_CK(ttk::sumsq(carry.p, W64, crow * ccol, d_carry2 + s, ws.p, st), "carry sum of squares");
    TT_RED(d_carry2 + s, 1);
    cores[k - 1] = core.release();
    if (cfg.urv)
      out->ranks[k - 1] = r;
    else
      out->ranks[k] = r;
    // the carry becomes the next unfolding; the previous one is released
    cbuf.reset();
    if (s == 0) {
      conv.reset();
      staged.reset();
    }
    cbuf.p = carry.release();
    C = cbuf.as<W>();
    r_carry = r;
    r_prev = r;
  }
  // last core: the final carry (Alg. 3 step 8 / Alg. 1 step 8); a
  // partitioned one is gathered, every rank returns the whole core
  if (active) {
    const int64_t rl = r_carry;  // r_1 (URV) or r_{d-1} (ULV)
    const int64_t lb = (cfg.urv ? dl[0] : dl[d - 1]) * rl;
    Buf whole(&al), parts(&al);
    TT_ALLOC(whole, (size_t)lb * sh->nranks * sizeof(W));
    if (cfg.urv) {
      const tt_status sg = gather(cbuf.p, whole.p, lb * (int64_t)sizeof(W));
      if (sg != TT_OK) return sg;
    } else {
      TT_ALLOC(parts, (size_t)lb * sh->nranks * sizeof(W));
      const tt_status sg = gather(cbuf.p, parts.p, lb * (int64_t)sizeof(W));
      if (sg != TT_OK) return sg;
      TT_CK(ttk::unshard_cols(parts.p, whole.p, W64, sh->nranks, rl, 1, dl[d - 1], st),
            "interleave the gathered core");
    }
    cbuf.reset();
    cbuf.p = whole.release();
  }
  cores[cfg.urv ? 0 : d - 1] = cbuf.release();
  double h_carry2[TT_MAXD], h_tdirect[TT_MAXD];
  TT_CK(cudaMemcpyAsync(h_carry2, d_carry2, sizeof(double) * (d - 1), cudaMemcpyDeviceToHost, st), "tails");
  TT_CK(cudaMemcpyAsync(h_tdirect, d_tdirect, sizeof(double) * (d - 1), cudaMemcpyDeviceToHost, st),
        "direct tails");
  TT_CK(cudaMemcpyAsync(herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, st), "error word");
  {
    const double t0 = host_us();
    TT_CK(cudaStreamSynchronize(st), "final sync");
    g_hprof.sync_us += host_us() - t0;
  }
  tm.collect();
  if (*herr) return fail(TT_ETIMEOUT, "a bounded wait in a tensor-core kernel ran out");
  for (int s = 0; s < d - 1; ++s) {
    const int k = cfg.urv ? d - s : s + 1;
    const int u = cfg.urv ? k - 1 : k;
    const double t = ftail[s] >= 0.0 ? ftail[s] : has_direct[s] ? h_tdirect[s] : x2s[s] - h_carry2[s];
    out->tail_sq[u - 1] = t > 0.0 ? t : 0.0;
  }
  out->norm_sq = normA2;
  for (int k = 0; k < d; ++k) out->cores[k] = cores[k];
  guard.ok = true;
  return TT_OK;
}

tt_status validate(const void* A, int32_t dtype, int32_t d, const int64_t* dims, double eps,
                   const int64_t* fixed, const tt_opts& o, tt_result* out) {
  if (!A || !dims || !out) return fail(TT_EINVAL, "NULL argument");
  if (d < 2 || d > TT_MAXD) return fail(TT_EINVAL, "order d must be in [2, 16]");
  if (dtype != TT_F32 && dtype != TT_F64) return fail(TT_EINVAL, "dtype must be TT_F32 or TT_F64");
  double total = 1.0;
  for (int k = 0; k < d; ++k) {
    if (dims[k] < 1) return fail(TT_EINVAL, "every mode size must be >= 1");
    total *= (double)dims[k];
  }
  if (total > 4.0e18) return fail(TT_EINVAL, "tensor too large");
  if (fixed) {
    for (int k = 0; k < d - 1; ++k)
      if (fixed[k] < 1) return fail(TT_EINVAL, "fixed ranks must be >= 1");
  } else if (!(eps > 0.0) || !isfinite(eps)) {
    return fail(TT_EINVAL, "eps must be positive and finite");
  }
  if (o.oversample < 0 || o.oversample > 128) return fail(TT_EINVAL, "oversample must be in [0, 128]");
  if (o.l_full < 1 || o.l_full > ttk::kMaxSmall) return fail(TT_EINVAL, "l_full must be in [1, 256]");
  if (o.precision < TT_P_FP64 || o.precision > TT_P_MIXED) return fail(TT_EINVAL, "bad precision");
  if (o.small_precision < TT_SMALL_AUTO || o.small_precision > TT_SMALL_DF)
    return fail(TT_EINVAL, "bad small_precision");
  if (o.orth_precision < TT_SMALL_AUTO || o.orth_precision > TT_SMALL_DF)
    return fail(TT_EINVAL, "bad orth_precision");
  if (o.reverse != 0 && o.reverse != 1) return fail(TT_EINVAL, "reverse must be 0 or 1");
  if (o.power_iters < 0 || o.power_iters > 8) return fail(TT_EINVAL, "power_iters must be in [0, 8]");
  if (o.inner != TT_INNER_QLP && o.inner != TT_INNER_USVP && o.inner != TT_INNER_LURV)
    return fail(TT_EINVAL, "bad inner factor");
  if (o.usvp_iters < 0 || o.usvp_iters > 64) return fail(TT_EINVAL, "usvp_iters must be in [0, 64]");
  if (o.direct_tails != 0 && o.direct_tails != 1) return fail(TT_EINVAL, "direct_tails must be 0 or 1");
  if (o.lhat != TT_LHAT_FULL && o.lhat != TT_LHAT_L11) return fail(TT_EINVAL, "bad lhat");
  if (o.lhat == TT_LHAT_L11 && o.inner != TT_INNER_QLP)
    return fail(TT_EINVAL, "the L_11-only carry needs the pivoted QLP inner factor");
  if (o.weights) {
    double s = 0.0, s1 = 0.0;
    for (int k = 0; k < d - 1; ++k) {
      if (!(o.weights[k] > 0.0) || !isfinite(o.weights[k])) return fail(TT_EINVAL, "weights must be positive");
      s += o.weights[k] * o.weights[k];
      s1 += o.weights[k];
    }
    if (o.lhat == TT_LHAT_L11) {
      if (fabs(s1 - 1.0) > 1e-6) return fail(TT_EINVAL, "L_11-only weights must satisfy sum w_k = 1");
    } else if (fabs(s - 1.0) > 1e-6) {
      return fail(TT_EINVAL, "weights must satisfy sum w_k^2 = 1");
    }
  }
  return TT_OK;
}

// reverse = 1 (the Remark after Thm 3.2): the sweep factors the index-reversed
// tensor A'(i_d, ..., i_1) = A(i_1, ..., i_d) and its cores are read back as
// cores of A -- core k of A is core d+1-k of A' with its two rank axes
// swapped, so a right-to-left TT-URV of A' is a left-orthogonal TT of A.
// Unfolding k of A' is the transpose of unfolding d-k of A: per-unfolding
// weights, fixed ranks and results are mapped accordingly.
tt_status run_reversed(const void* A, int32_t dtype, int32_t d, const int64_t* dims, double eps,
                       const int64_t* fixed, SweepCfg cfg, tt_opts o, Alloc& al,
                       tt_result* out) {
  cudaStream_t st = al.st;
  const bool in64 = dtype == TT_F64;
  const size_t el = in64 ? 8 : 4;
  int64_t total = 1;
  for (int k = 0; k < d; ++k) total *= dims[k];
  Buf staged(&al), rev(&al);
  const void* src = A;
  if (host_pointer(A)) {
    TT_ALLOC(staged, (size_t)total * el);
    TT_CK(cudaMemcpyAsync(staged.p, A, (size_t)total * el, cudaMemcpyHostToDevice, st), "copy input");
    src = staged.p;
  }
  TT_ALLOC(rev, (size_t)total * el);
  TT_CK(ttk::reverse_modes(src, rev.p, in64, d, dims, st), "reverse modes");
  staged.reset();
  int64_t rdims[TT_MAXD], rfixed[TT_MAXD];
  double rw[TT_MAXD];
  for (int k = 0; k < d; ++k) rdims[k] = dims[d - 1 - k];
  if (fixed)
    for (int k = 0; k < d - 1; ++k) rfixed[k] = fixed[d - 2 - k];
  if (o.weights) {
    for (int k = 0; k < d - 1; ++k) rw[k] = o.weights[d - 2 - k];
    o.weights = rw;
  }
  o.reverse = 0;
  tt_result r;
  const tt_status sr =
      o.precision == TT_P_FP64
          ? run_sweep<double>(rev.p, dtype, d, rdims, eps, fixed ? rfixed : nullptr, cfg, o, al, &r)
          : run_sweep<float>(rev.p, dtype, d, rdims, eps, fixed ? rfixed : nullptr, cfg, o, al, &r);
  if (sr != TT_OK) return sr;
  rev.reset();

  memset(out, 0, sizeof(*out));
  out->d = d;
  out->dtype = r.dtype;
  out->orth = 1 - r.orth;
  out->norm_sq = r.norm_sq;
  for (int k = 0; k < d; ++k) out->dims[k] = dims[k];
  for (int k = 0; k <= d; ++k) out->ranks[k] = r.ranks[d - k];
  for (int k = 0; k < d - 1; ++k) {
    out->tail_sq[k] = r.tail_sq[d - 2 - k];
    out->delta_sq[k] = r.delta_sq[d - 2 - k];
    out->sketch_l[k] = r.sketch_l[d - 2 - k];
    out->small_fp64[k] = r.small_fp64[d - 2 - k];
  }
  const bool c64 = r.dtype == TT_F64;
  const size_t cel = c64 ? 8 : 4;
  tt_status sc = TT_OK;
  for (int k = 0; k < d && sc == TT_OK; ++k) {
    const int kr = d - 1 - k;  // core k of A is core kr of A'
    const int64_t Ar = r.ranks[kr], Br = r.ranks[kr + 1];
    void* c = al.get((size_t)Ar * dims[k] * Br * cel);
    if (!c) {
      sc = fail(TT_ENOMEM, "allocator returned NULL for a core");
      break;
    }
    out->cores[k] = c;
    const cudaError_t e = ttk::swap_outer(r.cores[kr], c, c64, Ar, dims[k], Br, st);
    if (e != cudaSuccess) sc = cuda_fail(e, "core axes");
  }
  for (int k = 0; k < d; ++k) al.put(r.cores[k]);
  if (sc != TT_OK) {
    for (int k = 0; k < d; ++k) al.put(out->cores[k]);
    memset(out, 0, sizeof(*out));
  }
  return sc;
}

tt_status sweep_entry(const void* A, int32_t dtype, int32_t d, const int64_t* dims, double eps,
                      const int64_t* fixed, SweepCfg cfg, const tt_opts* opts, tt_alloc_fn alloc,
                      tt_free_fn free_fn, void* ctx, void* stream, tt_result* out,
                      const tt_shard* sh = nullptr) {
  g_err.clear();
  struct NvtxSweep {  // one NVTX range around the whole sweep
    NvtxSweep() { nvtxRangePushA("ttutv sweep"); }
    ~NvtxSweep() { nvtxRangePop(); }
  } nvtx_sweep;
  tt_opts o;
  tt_opts_default(&o);
  if (opts) o = *opts;
  tt_status v = validate(A, dtype, d, dims, eps, fixed, o, out);
  if (v != TT_OK) return v;
  if ((alloc == nullptr) != (free_fn == nullptr))
    return fail(TT_EINVAL, "alloc and free must both be given or both be NULL");
  if (sh) {
    if (sh->nranks < 1 || sh->rank < 0 || sh->rank >= sh->nranks)
      return fail(TT_EINVAL, "shard: rank must be in [0, nranks)");
    const int pm = cfg.urv ? 0 : d - 1;
    if (dims[pm] % sh->nranks != 0)
      return fail(TT_EINVAL, "shard: the partitioned mode must split into equal slabs");
    if (sh->nranks > 1 && (!sh->allreduce || !sh->allgather))
      return fail(TT_EINVAL, "shard: all-reduce and all-gather callbacks are required");
    if (o.reverse) return fail(TT_EUNSUPPORTED, "shard: the reversed sweep is not partitioned");
    if (cfg.svd) return fail(TT_EUNSUPPORTED, "shard: TT-SVD is not partitioned");
  }
  Alloc al{alloc, free_fn, ctx, (cudaStream_t)stream};
  g_hprof = HostProf();
  const double t0 = host_us();
  const uint64_t l0 = ttk::launches();
  tt_status st;
  if (o.reverse)
    st = run_reversed(A, dtype, d, dims, eps, fixed, cfg, o, al, out);
  else if (o.precision == TT_P_FP64)
    st = run_sweep<double>(A, dtype, d, dims, eps, fixed, cfg, o, al, out, sh);
  else
    st = run_sweep<float>(A, dtype, d, dims, eps, fixed, cfg, o, al, out, sh);
  if (host_prof())
    fprintf(stderr, "[ttutv] host: wall %.1f us, blocked in syncs %.1f us, allocator %.1f us (%d calls), %llu launches\n",
            host_us() - t0, g_hprof.sync_us, g_hprof.alloc_us, g_hprof.nalloc,
            (unsigned long long)(ttk::launches() - l0));
  return st;
}

}  // namespace

namespace ttk {
void set_last_error(const char* msg) { g_err = msg; }
TT_BOUNDS_READER(bounds_driver)
}  // namespace ttk

extern "C" {

void tt_opts_default(tt_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->precision = TT_P_FP32;
  o->small_precision = TT_SMALL_AUTO;
  o->oversample = 16;
  o->l_full = 256;
  o->seed = 0;
  o->weights = nullptr;
  o->orth_precision = TT_SMALL_AUTO;
  o->phase_ms = nullptr;
  o->inner = TT_INNER_QLP;
  o->usvp_iters = 8;
}

tt_status tt_utv(const void* A, int32_t dtype, int32_t d, const int64_t* dims, double eps,
                 const int64_t* fixed_ranks, int32_t variant, int32_t direction,
                 const tt_opts* opts, tt_alloc_fn alloc, tt_free_fn free_fn, void* alloc_ctx,
                 void* stream, tt_result* out) {
  // The inner factor is a pivoted QLP, C ~ (Q_1 Pi_2) L (Pi_1 Q_2)^T: a ULV
  // form of C whose URV form is the QR of L.  A right-to-left TT-ULV that
  // keeps the middle block [L_11; L_21] (the appendix's first case of Alg. 4)
  // carries C V_1 with error ||L_22||^2 -- exactly the right-to-left TT-URV;
  // mirrored, a left-to-right TT-URV keeping [R_11 R_12] is the left-to-right
  // TT-ULV.  Both pairings therefore run those sweeps.  Alg. 4 as printed
  // keeps L_11 alone (tt_opts.lhat = TT_LHAT_L11): its carry U_1 L_11 is
  // formed from the QLP's factors by the small kernel (T with C T = U_1 L_11).
  if (variant != TT_URV && variant != TT_ULV) return fail(TT_EINVAL, "bad variant");
  if (direction != TT_RL && direction != TT_LR) return fail(TT_EINVAL, "bad direction");
  const bool l11 = opts && opts->lhat == TT_LHAT_L11;
  if (l11 && !(variant == TT_ULV && direction == TT_RL))
    return fail(TT_EINVAL, "the L_11-only carry is Alg. 4: TT-ULV right-to-left");
  SweepCfg cfg{direction == TT_RL, false};
  cfg.l11 = l11;
  return sweep_entry(A, dtype, d, dims, eps, fixed_ranks, cfg, opts, alloc, free_fn, alloc_ctx,
                     stream, out);
}

tt_status tt_utv_sharded(const void* A_local, int32_t dtype, int32_t d, const int64_t* dims,
                         double eps, const int64_t* fixed_ranks, int32_t variant, int32_t direction,
                         const tt_opts* opts, tt_alloc_fn alloc, tt_free_fn free_fn, void* alloc_ctx,
                         void* stream, const tt_shard* shard, tt_result* out) {
  if (!shard) return fail(TT_EINVAL, "NULL shard");
  if (variant != TT_URV && variant != TT_ULV) return fail(TT_EINVAL, "bad variant");
  if (direction != TT_RL && direction != TT_LR) return fail(TT_EINVAL, "bad direction");
  const bool l11 = opts && opts->lhat == TT_LHAT_L11;
  if (l11 && !(variant == TT_ULV && direction == TT_RL))
    return fail(TT_EINVAL, "the L_11-only carry is Alg. 4: TT-ULV right-to-left");
  SweepCfg cfg{direction == TT_RL, false};
  cfg.l11 = l11;
  return sweep_entry(A_local, dtype, d, dims, eps, fixed_ranks, cfg, opts, alloc, free_fn, alloc_ctx,
                     stream, out, shard);
}

tt_status tt_svd(const void* A, int32_t dtype, int32_t d, const int64_t* dims, double eps,
                 const int64_t* fixed_ranks, int32_t direction, const tt_opts* opts,
                 tt_alloc_fn alloc, tt_free_fn free_fn, void* alloc_ctx, void* stream,
                 tt_result* out) {
  if (direction != TT_RL && direction != TT_LR) return fail(TT_EINVAL, "bad direction");
  if (opts && opts->lhat == TT_LHAT_L11) return fail(TT_EINVAL, "TT-SVD has no L_11-only carry");
  SweepCfg cfg{direction == TT_RL, true};
  return sweep_entry(A, dtype, d, dims, eps, fixed_ranks, cfg, opts, alloc, free_fn, alloc_ctx,
                     stream, out);
}

void tt_result_free(tt_result* r, tt_free_fn free_fn, void* alloc_ctx, void* stream) {
  if (!r) return;
  for (int k = 0; k < TT_MAXD; ++k) {
    if (!r->cores[k]) continue;
    if (free_fn)
      free_fn(r->cores[k], stream, alloc_ctx);
    else
      cudaFreeAsync(r->cores[k], (cudaStream_t)stream);
  }
  memset(r, 0, sizeof(*r));
}

size_t tt_full_work_bytes(int32_t d, const int64_t* dims, const int64_t* ranks, int32_t dtype) {
  if (d < 2 || d > TT_MAXD || !dims || !ranks) return 0;
  const size_t el = dtype == TT_F64 ? 8 : 4;
  int64_t rows = dims[0];
  size_t buf = 0, ws = 0;
  for (int k = 1; k < d; ++k) {
    const int64_t N = dims[k] * ranks[k + 1];
    ws = std::max(ws, dtype == TT_F64 ? ttk::gemm_ws_bytes<double>(rows, N, ranks[k], false)
                                      : ttk::gemm_ws_bytes<float>(rows, N, ranks[k], false));
    if (k < d - 1) buf = std::max(buf, (size_t)(rows * N) * el);
    rows *= dims[k];
  }
  buf = (buf + 255) & ~(size_t)255;
  return 2 * buf + ws + 256;
}

tt_status tt_full(int32_t d, const int64_t* dims, const int64_t* ranks, const void* const* cores,
                  int32_t dtype, void* out, void* work, void* stream) {
  g_err.clear();
  if (d < 2 || d > TT_MAXD || !dims || !ranks || !cores || !out || !work)
    return fail(TT_EINVAL, "bad argument");
  if (dtype != TT_F32 && dtype != TT_F64) return fail(TT_EINVAL, "bad dtype");
  if (ranks[0] != 1 || ranks[d] != 1) return fail(TT_EINVAL, "r_0 and r_d must be 1");
  for (int k = 0; k < d; ++k) {
    if (dims[k] < 1 || ranks[k + 1] < 1 || !cores[k]) return fail(TT_EINVAL, "bad dims/ranks/cores");
  }
  cudaStream_t st = (cudaStream_t)stream;
  const size_t el = dtype == TT_F64 ? 8 : 4;
  int64_t rows = dims[0];
  size_t buf = 0;
  {
    int64_t rr = dims[0];
    for (int k = 1; k < d - 1; ++k) {
      buf = std::max(buf, (size_t)(rr * dims[k] * ranks[k + 1]) * el);
      rr *= dims[k];
    }
  }
  buf = (buf + 255) & ~(size_t)255;
  char* b0 = (char*)work;
  char* b1 = b0 + buf;
  char* wsp = b1 + buf;
  const void* cur = cores[0];
  for (int k = 1; k < d; ++k) {
    const int64_t K = ranks[k], N = dims[k] * ranks[k + 1];
    void* nxt = (k == d - 1) ? out : (void*)((k & 1) ? b0 : b1);
    cudaError_t e;
    if (dtype == TT_F64)
      e = ttk::gemm<double>({(const double*)cur, K, true}, {(const double*)cores[k], N, true}, rows, N,
                            K, (double*)nxt, N, nullptr, false, nullptr, wsp, st);
    else
      e = ttk::gemm<float>({(const float*)cur, K, true}, {(const float*)cores[k], N, true}, rows, N,
                           K, (float*)nxt, N, nullptr, false, nullptr, wsp, st);
    if (e != cudaSuccess) return cuda_fail(e, "tt_full contraction");
    cur = nxt;
    rows *= dims[k];
  }
  return TT_OK;
}

}  // extern "C"

namespace {
// Orthogonalization of TT cores (Def. 2.2) by Cholesky-QR2 of each core's
// unfolding with FP64 Grams: left side, k = 1..d-1 in order, the unfolding
// [r_{k-1} I_k] x [r_k] of R_{k-1} G_k (R_0 = 1) is replaced by Q_k and
// R_k = Q_k^T (R_{k-1} G_k) is pushed into core k+1; right side, mirrored
// with the row unfoldings [r_{k-1}] x [I_k r_k], k = d..2.
struct OrthBufs {
  size_t g, s, r, core, cb, ws, sws, info, total;
};

template <typename W>
OrthBufs orth_layout(int32_t d, const int64_t* dims, const int64_t* ranks) {
  OrthBufs b{};
  int64_t rmax = 1, cmax = 1;
  size_t ws = 0;
  for (int k = 0; k < d; ++k) {
    rmax = std::max<int64_t>(rmax, std::max(ranks[k], ranks[k + 1]));
    cmax = std::max<int64_t>(cmax, ranks[k] * dims[k] * ranks[k + 1]);
  }
  for (int k = 0; k < d; ++k) {
    const int64_t m = ranks[k] * dims[k], r = ranks[k + 1];  // left unfolding
    const int64_t n = dims[k] * ranks[k + 1], q = ranks[k];   // right unfolding
    const int64_t shapes[9][4] = {{r, r, m, 1}, {m, r, r, 0}, {r, m, r, 0}, {r, r, m, 0},
                                  {q, q, n, 1}, {n, q, q, 0}, {q, n, q, 0}, {q, q, n, 0},
                                  {m, q, q, 0}};
    for (const auto& sh : shapes)
      ws = std::max(ws, ttk::gemm_ws_bytes<W>(sh[0], sh[1], sh[2], sh[3] != 0));
    if (k + 1 < d)  // the push into the next core
      ws = std::max(ws, ttk::gemm_ws_bytes<W>(r, dims[k + 1] * ranks[k + 2], r, false));
  }
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o += align256(bytes);
    return at;
  };
  b.g = take((size_t)rmax * rmax * sizeof(double));
  b.s = take((size_t)rmax * rmax * sizeof(W));
  b.r = take((size_t)rmax * rmax * sizeof(W));
  b.cb = align256((size_t)cmax * sizeof(W));
  b.core = take(3 * b.cb);
  b.ws = take(ws);
  b.sws = take(ttk::small_ws_bytes((int)rmax, true));
  b.info = take(sizeof(ttk::StepInfo));
  b.total = o;
  return b;
}

// Q of the Cholesky-QR2 of the columns of X (rows x r, element (i, j) at
// X(i, j) of the view), written through `store` (a row-major rows x r buffer
// or, for the right side, the transposed view).  Pass 1 shifts the Gram by
// 4 r u_64 of its trace so that a numerically rank-deficient unfolding stays
// factorable; pass 2 restores orthonormality to the data's rounding.
template <typename W>
cudaError_t cholqr2(ttk::Mat<W> X, int64_t rows, int64_t r, W* t0, ttk::Mat<W> out_view,
                    W* out_ptr, int64_t out_ld, char* base, const OrthBufs& b, cudaStream_t st) {
  double* G = reinterpret_cast<double*>(base + b.g);
  W* S = reinterpret_cast<W*>(base + b.s);
  void* ws = base + b.ws;
  ttk::SmallParams po;
  memset(&po, 0, sizeof(po));
  po.n = (int)r;
  po.mode = ttk::SM_ORTH;
  po.r_fixed = -1;
  po.r_cap = (int)r;
  const double u64 = 1.1102230246251565e-16;
  ttk::Mat<W> cur = X;
  for (int pass = 0; pass < 2; ++pass) {
    // G = cur^T cur: A(i, j) = cur(j, i)
    ttk::Mat<W> curT{cur.p, cur.ld, !cur.row};
    cudaError_t e = ttk::gemm<W>(curT, cur, r, r, rows, nullptr, 0, G, true, nullptr, ws, st, true);
    if (e != cudaSuccess) return e;
    po.shift_rel = pass == 0 ? 4.0 * (double)r * u64 : 0.0;
    po.piv_tol = pass == 0 ? 0.0 : 64.0 * (double)r * u64 * u64;
    e = ttk::small_factor(G, po, true, S, std::is_same<W, double>::value, (int)r, base + b.sws,
                          reinterpret_cast<ttk::StepInfo*>(base + b.info), st);
    if (e != cudaSuccess) return e;
    // next = cur S (rows x r)
    if (pass == 0) {
      e = ttk::gemm<W>(cur, {S, r, true}, rows, r, r, t0, r, nullptr, false, nullptr, ws, st);
      cur = {t0, r, true};
    } else if (out_view.row) {
      e = ttk::gemm<W>(cur, {S, r, true}, rows, r, r, out_ptr, out_ld, nullptr, false, nullptr, ws,
                       st);
    } else {
      // transposed output: out^T (r x rows) = S^T cur^T
      e = ttk::gemm<W>({S, r, false}, {cur.p, cur.ld, !cur.row}, r, rows, r, out_ptr, out_ld,
                       nullptr, false, nullptr, ws, st);
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename W>
tt_status orth_run(int32_t d, const int64_t* dims, const int64_t* ranks, const void* const* cores,
                   int32_t side, void* const* out, void* work, cudaStream_t st) {
  const OrthBufs b = orth_layout<W>(d, dims, ranks);
  char* base = (char*)work;
  W* R = reinterpret_cast<W*>(base + b.r);
  W* buf[3] = {reinterpret_cast<W*>(base + b.core), reinterpret_cast<W*>(base + b.core + b.cb),
               reinterpret_cast<W*>(base + b.core + 2 * b.cb)};
  void* ws = base + b.ws;
  cudaError_t e = cudaSuccess;
  if (side == 1) {  // left-orthogonal cores 1..d-1
    const W* M = (const W*)cores[0];
    for (int k = 0; k + 1 < d; ++k) {
      const int64_t m = ranks[k] * dims[k], r = ranks[k + 1];
      W* Q = (W*)out[k];
      e = cholqr2<W>({M, r, true}, m, r, buf[0], {Q, r, true}, Q, r, base, b, st);
      if (e != cudaSuccess) return cuda_fail(e, "orthogonalize: Cholesky-QR");
      // R_k = Q^T M, pushed into the next core
      e = ttk::gemm<W>({Q, r, false}, {M, r, true}, r, r, m, R, r, nullptr, false, nullptr, ws, st);
      if (e != cudaSuccess) return cuda_fail(e, "orthogonalize: R");
      const int64_t N = dims[k + 1] * ranks[k + 2];
      W* dst = (k + 2 == d) ? (W*)out[d - 1] : buf[1 + (k & 1)];
      e = ttk::gemm<W>({R, r, true}, {(const W*)cores[k + 1], N, true}, r, N, r, dst, N, nullptr,
                       false, nullptr, ws, st);
      if (e != cudaSuccess) return cuda_fail(e, "orthogonalize: push");
      M = dst;
    }
  } else {  // right-orthogonal cores 2..d
    const W* M = (const W*)cores[d - 1];
    for (int k = d - 1; k >= 1; --k) {
      const int64_t q = ranks[k], n = dims[k] * ranks[k + 1];
      W* Q = (W*)out[k];  // row-major q x n with orthonormal rows
      e = cholqr2<W>({M, n, false}, n, q, buf[0], {Q, n, false}, Q, n, base, b, st);
      if (e != cudaSuccess) return cuda_fail(e, "orthogonalize: Cholesky-QR");
      // R_k = M Q^T, pushed into the previous core
      e = ttk::gemm<W>({M, n, true}, {Q, n, false}, q, q, n, R, q, nullptr, false, nullptr, ws, st);
      if (e != cudaSuccess) return cuda_fail(e, "orthogonalize: R");
      const int64_t mrows = ranks[k - 1] * dims[k - 1];
      W* dst = (k == 1) ? (W*)out[0] : buf[1 + (k & 1)];
      e = ttk::gemm<W>({(const W*)cores[k - 1], q, true}, {R, q, true}, mrows, q, q, dst, q,
                       nullptr, false, nullptr, ws, st);
      if (e != cudaSuccess) return cuda_fail(e, "orthogonalize: push");
      M = dst;
    }
  }
  return TT_OK;
}

tt_status orth_validate(int32_t d, const int64_t* dims, const int64_t* ranks, int32_t dtype,
                        int32_t side) {
  if (d < 2 || d > TT_MAXD || !dims || !ranks) return fail(TT_EINVAL, "bad d, dims or ranks");
  if (dtype != TT_F32 && dtype != TT_F64) return fail(TT_EINVAL, "bad dtype");
  if (side != 0 && side != 1) return fail(TT_EINVAL, "side must be 0 (right) or 1 (left)");
  if (ranks[0] != 1 || ranks[d] != 1) return fail(TT_EINVAL, "r_0 and r_d must be 1");
  for (int k = 0; k < d; ++k) {
    if (dims[k] < 1 || ranks[k + 1] < 1) return fail(TT_EINVAL, "dims and ranks must be >= 1");
    if (ranks[k + 1] > ttk::kMaxSmall) return fail(TT_EINVAL, "ranks must be <= 256");
    if (side == 1 && k + 1 < d && ranks[k + 1] > ranks[k] * dims[k])
      return fail(TT_EINVAL, "r_k > r_{k-1} I_k: a left unfolding cannot be orthonormal");
    if (side == 0 && k >= 1 && ranks[k] > dims[k] * ranks[k + 1])
      return fail(TT_EINVAL, "r_{k-1} > I_k r_k: a right unfolding cannot be orthonormal");
  }
  return TT_OK;
}

}  // namespace

extern "C" {

size_t tt_orthogonalize_work_bytes(int32_t d, const int64_t* dims, const int64_t* ranks,
                                   int32_t dtype) {
  if (d < 2 || d > TT_MAXD || !dims || !ranks) return 0;
  return dtype == TT_F64 ? orth_layout<double>(d, dims, ranks).total
                         : orth_layout<float>(d, dims, ranks).total;
}

tt_status tt_orthogonalize(int32_t d, const int64_t* dims, const int64_t* ranks,
                           const void* const* cores, int32_t dtype, int32_t side, void* const* out,
                           void* work, void* stream) {
  g_err.clear();
  const tt_status v = orth_validate(d, dims, ranks, dtype, side);
  if (v != TT_OK) return v;
  if (!cores || !out || !work) return fail(TT_EINVAL, "NULL argument");
  for (int k = 0; k < d; ++k) {
    if (!cores[k] || !out[k]) return fail(TT_EINVAL, "NULL core");
    for (int j = 0; j < d; ++j)
      if (out[k] == cores[j]) return fail(TT_EINVAL, "out must not alias the input cores");
  }
  cudaStream_t st = (cudaStream_t)stream;
  return dtype == TT_F64 ? orth_run<double>(d, dims, ranks, cores, side, out, work, st)
                         : orth_run<float>(d, dims, ranks, cores, side, out, work, st);
}

}  // extern "C"

namespace {
// Slab of the first mode for tt_rse: as many slices as fit in 2^24 entries
// (at least one).
int64_t rse_slab_rows(int32_t d, const int64_t* dims) {
  int64_t p = 1;
  for (int k = 1; k < d; ++k) p *= dims[k];
  return std::max<int64_t>(1, std::min<int64_t>(dims[0], ((int64_t)1 << 24) / std::max<int64_t>(1, p)));
}
// Contraction scratch of tt_rse: the larger of a full slab's and the last
// (ragged) slab's -- a smaller product may split its inner dimension and so
// need more scratch.
size_t rse_full_work(int32_t d, const int64_t* dims, const int64_t* ranks, int32_t dtype,
                     int64_t s1) {
  int64_t sd[TT_MAXD];
  for (int k = 0; k < d; ++k) sd[k] = dims[k];
  sd[0] = s1;
  size_t w = tt_full_work_bytes(d, sd, ranks, dtype);
  const int64_t last = dims[0] % s1;
  if (last) {
    sd[0] = last;
    w = std::max(w, tt_full_work_bytes(d, sd, ranks, dtype));
  }
  return w;
}
}  // namespace

extern "C" {

size_t tt_rse_work_bytes(int32_t d, const int64_t* dims, const int64_t* ranks, int32_t dtype) {
  if (d < 2 || d > TT_MAXD || !dims || !ranks) return 0;
  const size_t el = dtype == TT_F64 ? 8 : 4;
  const int64_t s1 = rse_slab_rows(d, dims);
  int64_t n = s1;
  for (int k = 1; k < d; ++k) n *= dims[k];
  return align256((size_t)n * el) + align256(rse_full_work(d, dims, ranks, dtype, s1)) +
         align256(ttk::diff_sumsq_parts_bytes());
}

tt_status tt_rse(int32_t d, const int64_t* dims, const int64_t* ranks, const void* const* cores,
                 int32_t dtype, const void* A, void* work, double* out, void* stream) {
  g_err.clear();
  if (d < 2 || d > TT_MAXD || !dims || !ranks || !cores || !A || !work || !out)
    return fail(TT_EINVAL, "bad argument");
  if (dtype != TT_F32 && dtype != TT_F64) return fail(TT_EINVAL, "bad dtype");
  for (int k = 0; k < d; ++k)
    if (dims[k] < 1 || ranks[k + 1] < 1 || !cores[k]) return fail(TT_EINVAL, "bad dims/ranks/cores");
  if (ranks[0] != 1 || ranks[d] != 1) return fail(TT_EINVAL, "r_0 and r_d must be 1");
  cudaStream_t st = (cudaStream_t)stream;
  const bool f64 = dtype == TT_F64;
  const size_t el = f64 ? 8 : 4;
  const int64_t s1 = rse_slab_rows(d, dims);
  int64_t p = 1;
  for (int k = 1; k < d; ++k) p *= dims[k];
  int64_t sd[TT_MAXD];
  for (int k = 0; k < d; ++k) sd[k] = dims[k];
  sd[0] = s1;
  char* chunk = (char*)work;
  char* fw = chunk + align256((size_t)(s1 * p) * el);
  double* part = (double*)(fw + align256(rse_full_work(d, dims, ranks, dtype, s1)));
  const void* sc[TT_MAXD];
  for (int k = 1; k < d; ++k) sc[k] = cores[k];
  for (int64_t a = 0; a < dims[0]; a += s1) {
    sd[0] = std::min<int64_t>(s1, dims[0] - a);
    // core 1 is [1][I_1][r_1]: slices a .. a + sd[0] - 1 start at row a
    sc[0] = (const char*)cores[0] + (size_t)a * ranks[1] * el;
    const tt_status s = tt_full(d, sd, ranks, sc, dtype, chunk, fw, stream);
    if (s != TT_OK) return s;
    TT_CK(ttk::diff_sumsq((const char*)A + (size_t)(a * p) * el, chunk, f64, sd[0] * p, part, a == 0,
                          st),
          "difference sums");
  }
  TT_CK(ttk::sum_pairs(part, out, st), "difference totals");
  return TT_OK;
}

tt_status tt_sketch_matrix(int64_t rows, int64_t cols, uint64_t seed, int32_t step, int32_t dtype,
                           void* out, void* stream) {
  g_err.clear();
  if (rows < 0 || cols < 0 || !out || (dtype != TT_F32 && dtype != TT_F64))
    return fail(TT_EINVAL, "bad argument");
  cudaError_t e = ttk::fill_sketch(out, dtype == TT_F64, rows, cols, seed, (uint32_t)step, false,
                                   (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "tt_sketch_matrix");
  return TT_OK;
}

int64_t tt_bounds_violations(int32_t* first_line, int32_t reset) {
#ifdef TT_BOUNDS_CHECK
  unsigned int (*const readers[])(int*, bool) = {
      ttk::bounds_driver, ttk::bounds_gemm,       ttk::bounds_masked, ttk::bounds_misc,
      ttk::bounds_small,  ttk::bounds_small_fast, ttk::bounds_tc_gemm};
  int64_t total = 0;
  int32_t line = 0;
  for (auto rd : readers) {
    int l = 0;
    const unsigned int c = rd(&l, reset != 0);
    if (c && !line) line = l;
    total += c;
  }
  if (first_line) *first_line = line;
  return total;
#else
  (void)reset;
  if (first_line) *first_line = 0;
  return -1;
#endif
}

tt_status tt_wait_selftest(int32_t arrive, int64_t limit_ns, void* stream) {
  g_err.clear();
  if (limit_ns <= 0 || limit_ns > 10000000000ll) return fail(TT_EINVAL, "limit_ns in (0, 1e10]");
  cudaStream_t st = (cudaStream_t)stream;
  int* d_err = nullptr;
  TT_CK(cudaMallocAsync((void**)&d_err, sizeof(int), st), "selftest word");
  int h = 0;
  cudaError_t e = cudaMemsetAsync(d_err, 0, sizeof(int), st);
  if (e == cudaSuccess) e = ttk::wait_selftest(arrive != 0, (uint64_t)limit_ns, d_err, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(d_err, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "tt_wait_selftest");
  if (h) return fail(TT_ETIMEOUT, "the bounded wait ran out");
  return TT_OK;
}

uint64_t tt_kernel_launches(void) { return ttk::launches(); }

const char* tt_last_error(void) { return g_err.c_str(); }

const char* tt_version(void) { return "ttutv-gb300 0.1 (sm_103a)"; }

}  // extern "C"
