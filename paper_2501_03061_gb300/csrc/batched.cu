// Batched exchange: many independent V_x applications (each with its own orbital count, grid and
// kernel) in one call, the batched serving form of the fused pair-FFT path (Sec. IV-A1,
// Eq. vxdiag, applied per instance).
//
// Host runtime around the exchange kernels:
//   * autotuner: the pair-tile size of a grid (how many pair fields one FFT batch holds, which
//     sets the L2 footprint and the launch count), on 64^3 FP32 grids the kernel family (the
//     launch-pipelined TMA kernels or the compile-time tile kernels), and for the compile-time
//     kernels in FP32 the CTA size of their FFT tile kernels (128, 256 or 512 threads) are picked
//     by timing candidates (budgets of 12 MiB to 512 MiB) on the first item of that grid (its
//     first min(N, 32) orbitals) and kept in the context;
//   * concurrent branches: items are dealt to `batch_streams` streams (longest first, by pair
//     FFTs x grid points), each with its own scratch buffers, forked from and joined back to the
//     caller's stream with events, so the small items' kernels fill the tails of the large ones';
//   * CUDA graphs: the first call with a given item set runs eagerly once (this sizes every
//     workspace, builds schedules and tables and encodes nothing that later changes), then the
//     whole batch is captured on a context-owned stream into one graph, which this and every
//     later call with the same item set replays with a single launch;
//   * device error words (bounded TMA waits) are zeroed once at the start of the batch and read
//     once after it, instead of after every item.
#include <algorithm>
#include <cstdio>
#include <string>

#include "fft_fixed.cuh"
#include "internal.h"

namespace pt {

namespace {

struct GraphHolder {
  cudaGraphExec_t exec = nullptr;
  size_t nodes = 0;
  long long pairs = 0;
  ~GraphHolder() {
    if (exec) cudaGraphExecDestroy(exec);
  }
};

std::string grid_key(const pt_grid& g, pt_precision prec) {
  char b[96];
  snprintf(b, sizeof(b), "tune:%d:%d:%d:%d", g.nx, g.ny, g.nz, int(prec));
  return b;
}

struct Tuned {
  size_t budget;
  int engine;  // exchange64_engine for 64^3 FP32 grids (0 or 1); ignored elsewhere
  int ft;      // threads per CTA of the compile-time tile kernels
};

// Pick the pair-field budget (and the 64^3 engine) for the grid of `it` by timing candidates
// (cached per grid).
Tuned tuned_budget(pt_ctx* ctx, const pt_exchange_item& it, pt_precision prec, cudaStream_t st) {
  const std::string key = grid_key(it.grid, prec);
  auto c = ctx->caches.find(key);
  if (c != ctx->caches.end()) return *std::static_pointer_cast<Tuned>(c->second);
  const size_t field = ng_of(it.grid) * elem_bytes(prec);
  const int nt = std::min(it.N, 32);
  void* out = ctx->get("tune_out", size_t(nt) * field);
  cudaEvent_t e0, e1;
  PT_CUDA_CHECK(cudaEventCreate(&e0));
  PT_CUDA_CHECK(cudaEventCreate(&e1));
  Tuned best{ctx->scratch_budget, ctx->exchange64_engine == 1 ? 1 : 0, ctx->fft_threads};
  float best_ms = 1e30f;
  const size_t mib = size_t(1) << 20;
  const size_t cands[] = {12 * mib, 24 * mib, 48 * mib, 96 * mib, 192 * mib, 512 * mib};
  const bool two_engines = prec != PT_FP64 && exchange64_applies(it.grid);
  const bool fixed = fixed_cubic(it.grid);
  const int saved_engine = ctx->exchange64_engine, saved_ft = ctx->fft_threads;
  struct Variant {
    int engine, ft;
  };
  // the TMA pipeline (64^3 FP32 only), then the compile-time kernels with each CTA size (FP32) or 256
  std::vector<Variant> variants;
  if (two_engines) variants.push_back({0, saved_ft});
  const int fts[3] = {256, 128, 512};
  const int nft = (fixed && prec != PT_FP64) ? 3 : 1;
  for (int q = 0; q < nft; ++q) variants.push_back({two_engines ? 1 : saved_engine, fts[q]});
  try {
    for (const Variant& var : variants) {
      const int engine = var.engine;
      int last_b = -1;
      ctx->exchange64_engine = engine;
      ctx->fft_threads = var.ft;
      for (size_t cand : cands) {
        // candidates that give the same pair tile are the same schedule
        int b = std::min(nt, int(std::floor(std::sqrt(double(std::max<size_t>(1, cand / field))))));
        if (two_engines && engine == 0) b = std::min(b, kExchange64MaxTile);
        if (b == last_b) continue;
        last_b = b;
        ctx->budget_override = cand;
        exchange(ctx, it.src, it.occ, nt, nullptr, nt, out, it.grid, it.kernel, prec, st);  // builds the schedule
        PT_CUDA_CHECK(cudaEventRecord(e0, st));
        for (int r = 0; r < 2; ++r)
          exchange(ctx, it.src, it.occ, nt, nullptr, nt, out, it.grid, it.kernel, prec, st);
        PT_CUDA_CHECK(cudaEventRecord(e1, st));
        PT_CUDA_CHECK(cudaEventSynchronize(e1));
        float ms = 0.f;
        PT_CUDA_CHECK(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best_ms) {
          best_ms = ms;
          best = Tuned{cand, engine, var.ft};
        }
      }
    }
  } catch (...) {
    ctx->budget_override = 0;
    ctx->exchange64_engine = saved_engine;
    ctx->fft_threads = saved_ft;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    throw;
  }
  ctx->budget_override = 0;
  ctx->exchange64_engine = saved_engine;
  ctx->fft_threads = saved_ft;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!two_engines) best.engine = saved_engine;
  ctx->caches[key] = std::make_shared<Tuned>(best);
  return best;
}

// Items dealt to branches longest first (work ~ pair FFTs x grid points), each branch to the
// currently lightest one; the same assignment in the eager pass and in the capture.
std::vector<int> assign_branches(const pt_exchange_item* items, int count, int nb) {
  std::vector<int> order(count), branch(count, 0);
  std::vector<double> work(count), load(nb, 0.0);
  for (int k = 0; k < count; ++k) {
    const double m = items[k].tgt ? items[k].M : items[k].N;
    const double pairs = items[k].tgt ? double(items[k].N) * m : 0.5 * m * (m + 1);
    work[k] = pairs * double(ng_of(items[k].grid));
    order[k] = k;
  }
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work[a] > work[b]; });
  for (int k : order) {
    const int b = int(std::min_element(load.begin(), load.end()) - load.begin());
    branch[k] = b;
    load[b] += work[k];
  }
  return branch;
}

struct TagGuard {
  pt_ctx* ctx;
  int engine, ft;
  ~TagGuard() {
    ctx->scratch_tag.clear();
    ctx->budget_override = 0;
    ctx->exchange64_engine = engine;
    ctx->fft_threads = ft;
  }
};

long long run_items(pt_ctx* ctx, const pt_exchange_item* items, int count, const std::vector<Tuned>& tuned,
                    pt_precision prec, cudaStream_t st) {
  long long pairs = 0;
  TagGuard guard{ctx, ctx->exchange64_engine, ctx->fft_threads};
  const int nb = std::max(1, std::min(ctx->batch_streams, count));
  auto one = [&](int k, cudaStream_t s) {
    const pt_exchange_item& it = items[k];
    ctx->budget_override = tuned[k].budget;
    if (prec != PT_FP64 && exchange64_applies(it.grid)) ctx->exchange64_engine = tuned[k].engine;
    ctx->fft_threads = tuned[k].ft;
    pairs += exchange(ctx, it.src, it.occ, it.N, it.tgt, it.tgt ? it.M : it.N, it.out, it.grid, it.kernel, prec, s);
    ctx->exchange64_engine = guard.engine;
    ctx->fft_threads = guard.ft;
  };
  if (nb == 1) {
    for (int k = 0; k < count; ++k) one(k, st);
    return pairs;
  }
  while (int(ctx->side_streams.size()) < nb) {
    cudaStream_t s = nullptr;
    PT_CUDA_CHECK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    ctx->side_streams.push_back(s);
  }
  const std::vector<int> branch = assign_branches(items, count, nb);
  std::vector<cudaEvent_t> ev(nb + 1, nullptr);
  for (auto& e : ev) PT_CUDA_CHECK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  struct EvGuard {
    std::vector<cudaEvent_t>& v;
    ~EvGuard() {
      for (auto e : v)
        if (e) cudaEventDestroy(e);
    }
  } evg{ev};
  PT_CUDA_CHECK(cudaEventRecord(ev[nb], st));  // fork
  for (int b = 0; b < nb; ++b) {
    cudaStream_t s = ctx->side_streams[b];
    PT_CUDA_CHECK(cudaStreamWaitEvent(s, ev[nb], 0));
    ctx->scratch_tag = "#" + std::to_string(b);
    for (int k = 0; k < count; ++k)
      if (branch[k] == b) one(k, s);
    PT_CUDA_CHECK(cudaEventRecord(ev[b], s));
  }
  ctx->scratch_tag.clear();
  for (int b = 0; b < nb; ++b) PT_CUDA_CHECK(cudaStreamWaitEvent(st, ev[b], 0));  // join
  return pairs;
}

std::string batch_key(const pt_exchange_item* items, int count, pt_precision prec, const std::vector<Tuned>& tuned,
                      int streams) {
  std::string k = "graph:" + std::to_string(int(prec)) + ":" + std::to_string(count) + ":" + std::to_string(streams);
  char b[256];
  for (int i = 0; i < count; ++i) {
    const pt_exchange_item& it = items[i];
    snprintf(b, sizeof(b), "|%p,%p,%d,%p,%d,%p,%d,%d,%d,%.17g,%.17g,%.17g,%d,%.17g,%.17g,%zu,%d,%d", it.src,
             static_cast<const void*>(it.occ), it.N, it.tgt, it.M, it.out, it.grid.nx, it.grid.ny, it.grid.nz,
             it.grid.L[0], it.grid.L[1], it.grid.L[2], it.kernel.type, it.kernel.mu, it.kernel.g0, tuned[i].budget,
             tuned[i].engine, tuned[i].ft);
    k += b;
  }
  return k;
}

struct DeferGuard {
  pt_ctx* ctx;
  explicit DeferGuard(pt_ctx* c) : ctx(c) { ctx->defer_checks = true; }
  ~DeferGuard() {
    ctx->defer_checks = false;
    ctx->budget_override = 0;
  }
};

}  // namespace

long long exchange_batched(pt_ctx* ctx, const pt_exchange_item* items, int count, pt_precision prec,
                           cudaStream_t st, size_t* graph_nodes) {
  if (graph_nodes) *graph_nodes = 0;
  std::vector<Tuned> tuned(count, Tuned{ctx->scratch_budget, ctx->exchange64_engine == 1 ? 1 : 0, ctx->fft_threads});
  if (ctx->autotune)
    for (int k = 0; k < count; ++k) tuned[k] = tuned_budget(ctx, items[k], prec, st);
  int* err = static_cast<int*>(ctx->get("exchange_err", sizeof(int)));
  const std::string key = batch_key(items, count, prec, tuned, std::min(ctx->batch_streams, count));
  auto c = ctx->caches.find(key);
  if (ctx->use_graphs && c != ctx->caches.end()) {
    auto g = std::static_pointer_cast<GraphHolder>(c->second);
    PT_CUDA_CHECK(cudaGraphLaunch(g->exec, st));
    exchange_check(ctx, st);
    if (graph_nodes) *graph_nodes = g->nodes;
    return g->pairs;
  }
  long long pairs = 0;
  {
    // eager pass: sizes every workspace and builds every schedule and table the capture will use
    DeferGuard dg(ctx);
    PT_CUDA_CHECK(cudaMemsetAsync(err, 0, sizeof(int), st));
    pairs = run_items(ctx, items, count, tuned, prec, st);
  }
  exchange_check(ctx, st);
  if (!ctx->use_graphs) return pairs;
  if (!ctx->cap_stream) PT_CUDA_CHECK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
  const size_t held_before = ctx->held;
  cudaGraph_t graph = nullptr;
  {
    DeferGuard dg(ctx);
    PT_CUDA_CHECK(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
    try {
      PT_CUDA_CHECK(cudaMemsetAsync(err, 0, sizeof(int), ctx->cap_stream));
      run_items(ctx, items, count, tuned, prec, ctx->cap_stream);
    } catch (...) {
      cudaGraph_t g2 = nullptr;
      cudaStreamEndCapture(ctx->cap_stream, &g2);
      if (g2) cudaGraphDestroy(g2);
      cudaGetLastError();
      throw;
    }
    PT_CUDA_CHECK(cudaStreamEndCapture(ctx->cap_stream, &graph));
  }
  if (ctx->held != held_before) {
    cudaGraphDestroy(graph);
    fail(PT_CUDA, "batched exchange: a workspace changed during graph capture");
  }
  auto holder = std::make_shared<GraphHolder>();
  holder->pairs = pairs;
  PT_CUDA_CHECK(cudaGraphGetNodes(graph, nullptr, &holder->nodes));
  const cudaError_t ie = cudaGraphInstantiate(&holder->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) {
    cudaGetLastError();
    fail(PT_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ie));
  }
  // at most a few graphs per context: drop the others before keeping this one
  int ngraphs = 0;
  for (auto it = ctx->caches.begin(); it != ctx->caches.end();) {
    if (it->first.rfind("graph:", 0) == 0 && ++ngraphs > 3) it = ctx->caches.erase(it);
    else ++it;
  }
  ctx->caches[key] = holder;
  if (graph_nodes) *graph_nodes = holder->nodes;
  return pairs;
}

}  // namespace pt
