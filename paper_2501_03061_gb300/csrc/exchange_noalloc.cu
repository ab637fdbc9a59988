// pt_apply_exchange_noalloc: the exchange V_x tgt computed without any device allocation.
//
// Who needs it: callers that cannot call cudaMalloc while they run this code — for example a
// host application that has handed the whole device memory to its own pool allocator (a
// cudaMalloc from this library would fail or break its accounting), or a latency-critical loop
// that must not pay the implicit device synchronisation of cudaMalloc/cudaFree.  The regular
// entry point allocates its workspace (pair scratch, tables, schedules) on first use.
//
// Here every device buffer the computation needs beyond the caller's inputs and outputs lives in
// file-scope static __device__ arrays of fixed size, held by every GPU that loads the library
// until the process exits:
//   pair-field scratch  NOALLOC_SCRATCH_BYTES (32 MiB)
//   K(G)/Ng table       64^3 doubles (2 MiB)
//   twiddles, one batch's pair/target/contribution lists (a few tens of KiB)
// The arrays become resident when the CUDA runtime loads this library's device code on a GPU;
// under lazy module loading that can be inside the first call, so a caller that gives all free
// device memory to its own pool makes one call first.
// In host code the names of these arrays are host-side stand-ins, not device addresses, so the
// first call on each device (with that device current) fetches their device addresses with
// cudaGetSymbolAddress and keeps them; make that first call before any stream capture.
// Tables and schedules are written with stream-ordered copies; the generic three-pass exchange
// kernels then run on the static buffers.  All calls share the arrays and the last call's
// contents stay there: calls that overlap on the GPU (different streams or host threads) race.
// Nothing needs clearing: every pair field is written before it is read, pairs whose
// occupations are all zero are skipped on both sides, and each output orbital is written, not
// accumulated, by its first batch.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>

#include "exchange_sched.h"
#include "fft.cuh"
#include "internal.h"

namespace pt {

namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = size_t(32) << 20;
constexpr int NOALLOC_MAX_ORB = 1024;          // N and M
constexpr int NOALLOC_MAX_TILE = 32;           // pair tile side B
constexpr int NOALLOC_MAX_PAIRS = NOALLOC_MAX_TILE * NOALLOC_MAX_TILE;
constexpr int NOALLOC_MAX_TGTS = 2 * NOALLOC_MAX_TILE;
constexpr int NOALLOC_MAX_CONS = 2 * NOALLOC_MAX_PAIRS;
constexpr int NOALLOC_MAX_NG = kMaxDim * kMaxDim * kMaxDim;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];
static __device__ __align__(256) double g_noalloc_ktab[NOALLOC_MAX_NG];
static __device__ __align__(256) double g_noalloc_tw[2 * 3 * kMaxDim];
static __device__ __align__(256) PairDesc g_noalloc_pairs[NOALLOC_MAX_PAIRS];
static __device__ __align__(256) TargetDesc g_noalloc_tgts[NOALLOC_MAX_TGTS];
static __device__ __align__(256) Contrib g_noalloc_cons[NOALLOC_MAX_CONS];

struct DeviceAddrs {
  bool ready = false;
  void* scratch = nullptr;
  void* ktab = nullptr;
  void* tw = nullptr;
  PairDesc* pairs = nullptr;
  TargetDesc* tgts = nullptr;
  Contrib* cons = nullptr;
  std::string table_key;  // grid/kernel/precision whose tables the arrays currently hold
};

std::mutex g_noalloc_mutex;
DeviceAddrs g_noalloc_dev[64];

void symbol_addr(void** p, const void* sym, const char* what) {
  const cudaError_t e = cudaGetSymbolAddress(p, sym);
  if (e != cudaSuccess) fail(PT_CUDA, std::string("cudaGetSymbolAddress(") + what + "): " + cudaGetErrorString(e));
}

DeviceAddrs& device_addrs(int dev) {
  if (dev < 0 || dev >= 64) fail(PT_INVALID_ARG, "device index out of range");
  DeviceAddrs& a = g_noalloc_dev[dev];
  if (!a.ready) {
    void* p = nullptr;
    symbol_addr(&a.scratch, g_noalloc_scratch, "scratch");
    symbol_addr(&a.ktab, g_noalloc_ktab, "kernel table");
    symbol_addr(&a.tw, g_noalloc_tw, "twiddles");
    symbol_addr(&p, g_noalloc_pairs, "pairs");
    a.pairs = static_cast<PairDesc*>(p);
    symbol_addr(&p, g_noalloc_tgts, "targets");
    a.tgts = static_cast<TargetDesc*>(p);
    symbol_addr(&p, g_noalloc_cons, "contributions");
    a.cons = static_cast<Contrib*>(p);
    a.ready = true;
  }
  return a;
}

int wrapped(int i, int n) { return i < (n + 1) / 2 ? i : i - n; }

template <class T>
void fill_tables(DeviceAddrs& a, const pt_grid& g, const pt_kernel& k, cudaStream_t st) {
  char key[200];
  snprintf(key, sizeof(key), "%d:%d:%d:%.17g:%.17g:%.17g:%d:%.17g:%.17g:%zu", g.nx, g.ny, g.nz, g.L[0], g.L[1],
           g.L[2], k.type, k.mu, k.g0, sizeof(T));
  if (a.table_key == key) return;
  const int ns[3] = {g.nx, g.ny, g.nz};
  std::vector<cx<T>> tw;
  for (int ax = 0; ax < 3; ++ax)
    for (int i = 0; i < ns[ax]; ++i) {
      const double ang = -2.0 * M_PI * double(i) / double(ns[ax]);
      tw.push_back(cx<T>{T(std::cos(ang)), T(std::sin(ang))});
    }
  const size_t ng = ng_of(g);
  std::vector<T> kt(ng);
  for (int z = 0; z < g.nz; ++z) {
    const double gz = 2.0 * M_PI * wrapped(z, g.nz) / g.L[2];
    for (int y = 0; y < g.ny; ++y) {
      const double gy = 2.0 * M_PI * wrapped(y, g.ny) / g.L[1];
      for (int x = 0; x < g.nx; ++x) {
        const double gx = 2.0 * M_PI * wrapped(x, g.nx) / g.L[0];
        kt[(size_t(z) * g.ny + y) * g.nx + x] = T(kernel_value(k, gx * gx + gy * gy + gz * gz) / double(ng));
      }
    }
  }
  // pageable-memory copies are staged before the call returns, so the vectors may go out of scope
  PT_CUDA_CHECK(cudaMemcpyAsync(a.tw, tw.data(), tw.size() * sizeof(cx<T>), cudaMemcpyHostToDevice, st));
  PT_CUDA_CHECK(cudaMemcpyAsync(a.ktab, kt.data(), kt.size() * sizeof(T), cudaMemcpyHostToDevice, st));
  a.table_key = key;
}

// One batch of the pair schedule: pairs (i, j), targets with their contributions (indices rebased
// to the batch).  Symmetric: B x B tiles I <= J with i <= j inside diagonal tiles.
struct Batch {
  std::vector<PairDesc> pairs;
  std::vector<TargetDesc> tgts;
  std::vector<Contrib> cons;
};

template <class T>
void run(const cx<T>* src, const double* occ, int N, const cx<T>* tgt, int M, cx<T>* out, const pt_grid& g,
         const pt_kernel& k, cudaStream_t st) {
  const bool sym = (tgt == nullptr);
  if (sym) {
    tgt = src;
    M = N;
  }
  if (N > NOALLOC_MAX_ORB || M > NOALLOC_MAX_ORB)
    fail(PT_INVALID_ARG, "pt_apply_exchange_noalloc: N and M are limited to 1024");
  const size_t ng = ng_of(g);
  const size_t field = ng * sizeof(cx<T>);
  if (ng > size_t(NOALLOC_MAX_NG) || field > NOALLOC_SCRATCH_BYTES)
    fail(PT_INVALID_ARG, "pt_apply_exchange_noalloc: grid exceeds the static scratch");
  int dev = 0;
  PT_CUDA_CHECK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  DeviceAddrs& a = device_addrs(dev);
  fill_tables<T>(a, g, k, st);
  const GridPlan gp = make_grid_plan(g);
  int B = int(std::floor(std::sqrt(double(NOALLOC_SCRATCH_BYTES / field))));
  B = std::max(1, std::min(std::min(B, NOALLOC_MAX_TILE), std::max(N, M)));
  std::vector<char> touched(M, 0);
  cx<T>* scratch = static_cast<cx<T>*>(a.scratch);
  auto flush = [&](Batch& b, std::map<int, std::vector<Contrib>>& per_t) {
    for (auto& kv : per_t) {
      TargetDesc td;
      td.t = kv.first;
      td.cbeg = int(b.cons.size());
      for (auto& c : kv.second) b.cons.push_back(c);
      td.cend = int(b.cons.size());
      td.first = touched[kv.first] ? 0 : 1;
      touched[kv.first] = 1;
      b.tgts.push_back(td);
    }
    PT_CUDA_CHECK(cudaMemcpyAsync(a.pairs, b.pairs.data(), b.pairs.size() * sizeof(PairDesc), cudaMemcpyHostToDevice,
                                  st));
    PT_CUDA_CHECK(
        cudaMemcpyAsync(a.tgts, b.tgts.data(), b.tgts.size() * sizeof(TargetDesc), cudaMemcpyHostToDevice, st));
    PT_CUDA_CHECK(
        cudaMemcpyAsync(a.cons, b.cons.data(), b.cons.size() * sizeof(Contrib), cudaMemcpyHostToDevice, st));
    exchange_batch_generic<T>(gp, src, tgt, occ, a.pairs, int(b.pairs.size()), a.tgts, int(b.tgts.size()), a.cons,
                              static_cast<const T*>(a.ktab), static_cast<const cx<T>*>(a.tw), scratch, out, st);
  };
  if (sym) {
    const int nb = (N + B - 1) / B;
    for (int J = 0; J < nb; ++J)
      for (int I = 0; I <= J; ++I) {
        Batch b;
        std::map<int, std::vector<Contrib>> per_t;
        const int i0 = I * B, i1 = std::min(N, i0 + B), j0 = J * B, j1 = std::min(N, j0 + B);
        for (int i = i0; i < i1; ++i)
          for (int j = (I == J ? i : j0); j < j1; ++j) {
            const int slot = int(b.pairs.size());
            b.pairs.push_back({i, j, i, i == j ? -1 : j});
            per_t[j].push_back({slot, i, i, 0});
            if (i != j) per_t[i].push_back({slot, j, j, 1});
          }
        flush(b, per_t);
      }
  } else {
    const int nbi = (N + B - 1) / B, nbj = (M + B - 1) / B;
    for (int J = 0; J < nbj; ++J)
      for (int I = 0; I < nbi; ++I) {
        Batch b;
        std::map<int, std::vector<Contrib>> per_t;
        const int i0 = I * B, i1 = std::min(N, i0 + B), j0 = J * B, j1 = std::min(M, j0 + B);
        for (int j = j0; j < j1; ++j)
          for (int i = i0; i < i1; ++i) {
            const int slot = int(b.pairs.size());
            b.pairs.push_back({i, j, i, -1});
            per_t[j].push_back({slot, i, i, 0});
          }
        flush(b, per_t);
      }
  }
}

}  // namespace

}  // namespace pt

extern "C" pt_status pt_apply_exchange_noalloc(const void* src, const double* occ, int N, const void* tgt, int M,
                                               void* out, const pt_grid* grid, const pt_kernel* kernel,
                                               pt_precision prec, void* stream) {
  try {
    pt::validate_grid(grid);
    if (!kernel || (kernel->type != 0 && kernel->type != 1) || (kernel->type == 1 && !(kernel->mu > 0)))
      pt::fail(PT_INVALID_ARG, "bad kernel");
    if (prec < PT_FP64 || prec > PT_FP32_TC_BF16) pt::fail(PT_INVALID_ARG, "unknown precision");
    if (N <= 0 || N > PT_MAX_ORBITALS || (tgt && (M <= 0 || M > PT_MAX_ORBITALS)) || !occ)
      pt::fail(PT_INVALID_ARG, "bad sizes or NULL occupations");
    pt::require_aligned(src, "src");
    pt::require_aligned(out, "out");
    if (tgt) pt::require_aligned(tgt, "tgt");
    if (out == src || (tgt && out == tgt)) pt::fail(PT_INVALID_ARG, "out must not alias src or tgt");
    auto st = static_cast<cudaStream_t>(stream);
    if (prec == PT_FP64)
      pt::run<double>(static_cast<const c128*>(src), occ, N, static_cast<const c128*>(tgt), M,
                      static_cast<c128*>(out), *grid, *kernel, st);
    else
      pt::run<float>(static_cast<const c64*>(src), occ, N, static_cast<const c64*>(tgt), M, static_cast<c64*>(out),
                     *grid, *kernel, st);
    return PT_OK;
  } catch (const pt::Error& e) {
    return e.code;
  } catch (...) {
    return PT_CUDA;
  }
}
