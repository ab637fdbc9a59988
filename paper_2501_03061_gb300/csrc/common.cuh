// Shared internals of the PT-IM library: complex arithmetic, the context with
// its workspace arena, error handling and launch accounting.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/ptim.h"

// ------------------------------------------------------------------------------------------
// complex numbers (interleaved re, im; 8- or 16-byte aligned for vector loads)
// ------------------------------------------------------------------------------------------
template <class T>
struct alignas(2 * sizeof(T)) cx {
  T re, im;
};

template <class T> __host__ __device__ __forceinline__ cx<T> mk(T a, T b) { return cx<T>{a, b}; }
template <class T> __host__ __device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <class T> __host__ __device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <class T> __host__ __device__ __forceinline__ cx<T> operator*(cx<T> a, T s) { return {a.re * s, a.im * s}; }
template <class T> __host__ __device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
// conj(a) * b
template <class T> __host__ __device__ __forceinline__ cx<T> cmulc(cx<T> a, cx<T> b) {
  return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
template <class T> __host__ __device__ __forceinline__ cx<T> conjc(cx<T> a) { return {a.re, -a.im}; }
// acc += a * b
template <class T> __host__ __device__ __forceinline__ void cfma(cx<T>& acc, cx<T> a, cx<T> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
}
// multiply by -i (forward) or +i (inverse)
template <bool INV, class T> __host__ __device__ __forceinline__ cx<T> rot90(cx<T> a) {
  return INV ? cx<T>{-a.im, a.re} : cx<T>{a.im, -a.re};
}
template <class T> __host__ __device__ __forceinline__ cx<T> czero() { return {T(0), T(0)}; }

using c64 = cx<float>;
using c128 = cx<double>;

template <class T> __host__ __device__ __forceinline__ cx<T> to_cx(c128 a) { return {T(a.re), T(a.im)}; }

// ------------------------------------------------------------------------------------------
// errors, launches
// ------------------------------------------------------------------------------------------
namespace pt {

extern std::atomic<long long> g_launches;

struct Error {
  pt_status code;
  std::string msg;
};

// Throw inside the library; the C ABI entry points catch and convert to pt_status.
[[noreturn]] void fail(pt_status code, const std::string& msg);
void check_cuda(cudaError_t e, const char* what);

#define PT_CUDA_CHECK(expr) ::pt::check_cuda((expr), #expr)

// Runs a set-up action (kernel attributes, constant-memory tables) once per CUDA device: both are
// per-device state, and the serving loop calls the library from several threads.
class DeviceOnce {
 public:
  template <class F>
  void operator()(F&& f) {
    int dev = 0;
    check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= 64) fail(PT_CUDA, "device index out of range");
    const uint64_t bit = uint64_t(1) << dev;
    std::lock_guard<std::mutex> lock(m_);
    if (done_ & bit) return;
    f();
    done_ |= bit;
  }

 private:
  std::mutex m_;
  uint64_t done_ = 0;
};
// Launch a kernel, count it, and surface launch-configuration errors immediately.
#define PT_LAUNCH(kernel, grid, block, smem, stream, ...)                          \
  do {                                                                            \
    kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);                   \
    ::pt::g_launches.fetch_add(1, std::memory_order_relaxed);                     \
    ::pt::check_cuda(cudaGetLastError(), #kernel);                                \
  } while (0)

// Programmatic dependent launch for chains of short dependent kernels (the N x N FP64 chains):
// the kernel may be launched while its predecessor on the stream still runs.  A kernel launched
// this way calls pdl_wait() before it reads anything an earlier kernel wrote (it returns once the
// predecessor has completed and its writes are visible; a no-op for a plain launch), then
// pdl_launch_dependents(), which lets the next link of the chain be launched; so at most two
// links are resident at a time.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

#define PT_LAUNCH_PDL(kernel, grid, block, smem, strm, ...)                        \
  do {                                                                            \
    cudaLaunchConfig_t cfg_{};                                                    \
    cfg_.gridDim = dim3(grid);                                                    \
    cfg_.blockDim = dim3(block);                                                  \
    cfg_.dynamicSmemBytes = (smem);                                               \
    cfg_.stream = (strm);                                                         \
    cudaLaunchAttribute at_[1];                                                   \
    at_[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;               \
    at_[0].val.programmaticStreamSerializationAllowed = 1;                        \
    cfg_.attrs = at_;                                                             \
    cfg_.numAttrs = 1;                                                            \
    ::pt::check_cuda(cudaLaunchKernelEx(&cfg_, kernel, __VA_ARGS__), #kernel);    \
    ::pt::g_launches.fetch_add(1, std::memory_order_relaxed);                     \
  } while (0)

// ------------------------------------------------------------------------------------------
// context and workspace
// ------------------------------------------------------------------------------------------
struct DevBuf {
  void* ptr = nullptr;
  size_t bytes = 0;
};

struct FftTables;  // per (grid, precision): twiddles, axis tables
struct KernelTable;
struct Schedule;

}  // namespace pt

struct pt_ctx {
  int device = 0;
  size_t budget = 0;
  size_t held = 0;
  int num_sms = 0;
  size_t max_smem_optin = 0;
  // bytes of pair fields per exchange batch (and of orbital fields per H batch); larger batches
  // cost less per pair even past L2 residency (fewer launches, traffic amortised over the tile)
  size_t scratch_budget = size_t(512) << 20;
  // bytes of pair fields per batch on the 64^3 FP32 TMA pipeline: its cost per pair falls with the
  // pair tile (fewer launches, W traffic amortised over more contributions), so it takes the
  // largest tile its parameter block holds rather than an L2-sized one
  size_t tma64_budget = size_t(512) << 20;
  int tc_gram = 0;     // option: FP32 form's Gram contractions on tensor cores (3xTF32) when 1
  int active_tc = 0;   // per call: 0 CUDA cores, 1 tensor cores 3xTF32, 2 tensor cores single TF32
  bool bf16_requested = false;  // per call: the BF16 form, whose contractions are not built
  double ptim_inner_kappa = 0.1;  // option: inner tolerance = max(tol, min(cap, kappa * midpoint move))
  double ptim_inner_cap = 1e-2;   // option: loosest inner tolerance (also that of the first outer iteration)
  int ptim_precond = 1;        // option: Anderson on the kinetically preconditioned inner map when 1
  int ptim_ace_warm = 1;       // option: a chained step's first outer pass uses the previous step's ACE
  int ptim_pw = 1;             // option: the step's orbital blocks as plane-wave coefficients when 1
  int ptim_sinv_mixed = 1;      // option: S^{-1} A from an FP32 factor refined in FP64 when 1
  int ptim_sinv_series = 1;    // option: S^{-1} A of the PT-IM inner iteration by a series in S - I when
                               // S is near the identity (1 cheapest form, 2 product form, 0 Cholesky only)
  bool ptim_warm_valid = false;  // "ptim_xi" holds the last ACE of the step whose output is fingerprinted
  std::string ptim_warm_key;     // sizes, grid, kernel and precision of that step
  unsigned long long ptim_warm_fp[2] = {0, 0};  // fingerprint of that step's output (phi, sigma)
  int ptim_q_n = 0;            // the "ptim_Q" buffer holds a complete unitary ptim_q_n x ptim_q_n basis
  // option: 64^3 FP32 exchange engine: 0 the launch-pipelined TMA kernel (roles A, B, C, D), 1 the
  // compile-time tile kernels, 2 one persistent cooperative launch per application
  // (exchange64_persist.cu), 3 the launch-pipelined TMA kernel with C fused into the accumulate
  int exchange64_engine = 0;
  int x64p_tile = 4;   // option: pair-tile side of the persistent engine's schedule
  int x64p_ring = 24;  // option: pair-field ring slots of the persistent engine (raised to tile pairs + 3 lag + 1)
  int x64p_lag = 2;    // option: waves between the A, B, C and D stages of a pair in the persistent engine
  int tc_gram_wide = 1;  // option: 64 x 128 tensor-core Gram tiles (and the fused two-product pass) when 1
  int tc_period = 2;   // option: K stages (32 floats each) accumulated in TMEM between readouts
  bool tc_err_clean = false;  // the tensor-core Gram's device error word exists and has been zeroed
  // batched exchange (batched.cu)
  int use_graphs = 1;          // option "graphs": replay repeated batches from captured CUDA graphs
  int autotune = 1;            // option "autotune": pick the pair-tile budget per grid by measurement
  size_t budget_override = 0;  // pair-field budget in force for the current batched call (0: scratch_budget)
  bool defer_checks = false;   // inside a batched call: device error words are checked once at the end
  cudaStream_t cap_stream = nullptr;  // non-default stream that graph captures are recorded on
  int batch_streams = 4;              // option: concurrent branches (streams) of a batched exchange call
  int fft_threads = 256;              // option: threads per CTA of the compile-time exchange tile kernels
  std::vector<cudaStream_t> side_streams;  // the branches' streams (created on first use)
  std::string scratch_tag;            // suffix of the exchange scratch names: one set per concurrent branch
  std::string tagged(const char* name) const { return std::string(name) + scratch_tag; }
  std::string err;
  std::map<std::string, pt::DevBuf> bufs;
  std::map<std::string, std::shared_ptr<void>> caches;  // keyed host-side caches of device tables

  // Grow-only named workspace.  The returned pointer stays valid until the next
  // get() of the same name with a larger size, or pt_trim.
  void* get(const std::string& name, size_t bytes);
  void release_all();
};

struct pt_ace {
  pt_ctx* ctx = nullptr;
  int N = 0;
  pt_grid grid{};
  pt_precision prec = PT_FP64;
  void* xi = nullptr;  // Ng x N, precision prec
  size_t bytes = 0;
};

namespace pt {

inline size_t elem_bytes(pt_precision p) { return p == PT_FP64 ? sizeof(c128) : sizeof(c64); }
inline bool is_fp32(pt_precision p) { return p != PT_FP64; }
inline size_t ng_of(const pt_grid& g) { return size_t(g.nx) * g.ny * g.nz; }
inline double dv_of(const pt_grid& g) { return g.L[0] * g.L[1] * g.L[2] / double(ng_of(g)); }

void validate_grid(const pt_grid* g);
void require_aligned(const void* p, const char* what);

}  // namespace pt
