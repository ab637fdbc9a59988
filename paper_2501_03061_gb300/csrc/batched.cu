// Batched exchange: many independent V_x applications (each with its own orbital count, grid and
// kernel) in one call, the batched serving form of the fused pair-FFT path (Sec. IV-A1,
// Eq. vxdiag, applied per instance).
//
// Host runtime around the exchange kernels:
//   * autotuner: the pair-tile size of a grid (how many pair fields one FFT batch holds, which
//     sets the L2 footprint and the launch count) is picked by timing candidate budgets of
//     12 MiB to 512 MiB on the first item of that grid (its first min(N, 32) orbitals) and kept
//     in the context;
//   * CUDA graphs: the first call with a given item set runs eagerly once (this sizes every
//     workspace, builds schedules and tables and encodes nothing that later changes), then the
//     whole batch is captured on a context-owned stream into one graph, which this and every
//     later call with the same item set replays with a single launch;
//   * device error words (bounded TMA waits) are zeroed once at the start of the batch and read
//     once after it, instead of after every item.
#include <algorithm>
#include <cstdio>
#include <string>

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

// Pick the pair-field budget for the grid of `it` by timing candidates (cached per grid).
size_t tuned_budget(pt_ctx* ctx, const pt_exchange_item& it, pt_precision prec, cudaStream_t st) {
  const std::string key = grid_key(it.grid, prec);
  auto c = ctx->caches.find(key);
  if (c != ctx->caches.end()) return *std::static_pointer_cast<size_t>(c->second);
  const size_t field = ng_of(it.grid) * elem_bytes(prec);
  const int nt = std::min(it.N, 32);
  void* out = ctx->get("tune_out", size_t(nt) * field);
  cudaEvent_t e0, e1;
  PT_CUDA_CHECK(cudaEventCreate(&e0));
  PT_CUDA_CHECK(cudaEventCreate(&e1));
  size_t best = ctx->scratch_budget;
  float best_ms = 1e30f;
  int last_b = -1;
  const size_t mib = size_t(1) << 20;
  const size_t cands[] = {12 * mib, 24 * mib, 48 * mib, 96 * mib, 192 * mib, 512 * mib};
  try {
    for (size_t cand : cands) {
      // candidates that give the same pair tile are the same schedule
      const int b = std::min(nt, int(std::floor(std::sqrt(double(std::max<size_t>(1, cand / field))))));
      if (b == last_b) continue;
      last_b = b;
      ctx->budget_override = cand;
      exchange(ctx, it.src, it.occ, nt, nullptr, nt, out, it.grid, it.kernel, prec, st);  // builds the schedule
      PT_CUDA_CHECK(cudaEventRecord(e0, st));
      for (int r = 0; r < 2; ++r) exchange(ctx, it.src, it.occ, nt, nullptr, nt, out, it.grid, it.kernel, prec, st);
      PT_CUDA_CHECK(cudaEventRecord(e1, st));
      PT_CUDA_CHECK(cudaEventSynchronize(e1));
      float ms = 0.f;
      PT_CUDA_CHECK(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best_ms) {
        best_ms = ms;
        best = cand;
      }
    }
  } catch (...) {
    ctx->budget_override = 0;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    throw;
  }
  ctx->budget_override = 0;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->caches[key] = std::make_shared<size_t>(best);
  return best;
}

long long run_items(pt_ctx* ctx, const pt_exchange_item* items, int count, const std::vector<size_t>& budgets,
                    pt_precision prec, cudaStream_t st) {
  long long pairs = 0;
  for (int k = 0; k < count; ++k) {
    const pt_exchange_item& it = items[k];
    ctx->budget_override = budgets[k];
    pairs += exchange(ctx, it.src, it.occ, it.N, it.tgt, it.tgt ? it.M : it.N, it.out, it.grid, it.kernel, prec, st);
  }
  ctx->budget_override = 0;
  return pairs;
}

std::string batch_key(const pt_exchange_item* items, int count, pt_precision prec, const std::vector<size_t>& budgets) {
  std::string k = "graph:" + std::to_string(int(prec)) + ":" + std::to_string(count);
  char b[256];
  for (int i = 0; i < count; ++i) {
    const pt_exchange_item& it = items[i];
    snprintf(b, sizeof(b), "|%p,%p,%d,%p,%d,%p,%d,%d,%d,%.17g,%.17g,%.17g,%d,%.17g,%.17g,%zu", it.src,
             static_cast<const void*>(it.occ), it.N, it.tgt, it.M, it.out, it.grid.nx, it.grid.ny, it.grid.nz,
             it.grid.L[0], it.grid.L[1], it.grid.L[2], it.kernel.type, it.kernel.mu, it.kernel.g0, budgets[i]);
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
  std::vector<size_t> budgets(count, ctx->scratch_budget);
  if (ctx->autotune)
    for (int k = 0; k < count; ++k) budgets[k] = tuned_budget(ctx, items[k], prec, st);
  int* err = static_cast<int*>(ctx->get("exchange_err", sizeof(int)));
  const std::string key = batch_key(items, count, prec, budgets);
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
    pairs = run_items(ctx, items, count, budgets, prec, st);
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
      run_items(ctx, items, count, budgets, prec, ctx->cap_stream);
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
