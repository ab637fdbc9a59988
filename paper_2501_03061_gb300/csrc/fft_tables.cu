// FFT plans and per-grid device tables (twiddles, per-axis |G|^2, the exchange kernel K(G)/Ng).
#include <cstring>

#include "fft.cuh"
#include "internal.h"

namespace pt {

bool make_axis_plan(int n, AxisPlan* ap) {
  if (n < 2 || n > kMaxDim) return false;
  std::memset(ap, 0, sizeof(*ap));
  ap->n = n;
  int rest = n, L = 1;
  const int radices[5] = {8, 4, 5, 3, 2};
  for (int r : radices) {
    while (rest % r == 0) {
      if (ap->nst >= kMaxStages) return false;
      ap->R[ap->nst] = r;
      ap->L[ap->nst] = L;
      ap->nst++;
      L *= r;
      rest /= r;
    }
  }
  return rest == 1;
}

GridPlan make_grid_plan(const pt_grid& g) {
  GridPlan gp;
  std::memset(&gp, 0, sizeof(gp));
  if (!make_axis_plan(g.nx, &gp.ax[0]) || !make_axis_plan(g.ny, &gp.ax[1]) || !make_axis_plan(g.nz, &gp.ax[2]))
    fail(PT_INVALID_ARG, "grid dimensions must be 2..64 and 2,3,5-smooth");
  gp.nx = g.nx;
  gp.ny = g.ny;
  gp.nz = g.nz;
  gp.pitch_x = (g.nx % 2 == 0) ? g.nx + 1 : g.nx;
  return gp;
}

void validate_grid(const pt_grid* g) {
  if (!g) fail(PT_INVALID_ARG, "grid is NULL");
  AxisPlan ap;
  if (!make_axis_plan(g->nx, &ap) || !make_axis_plan(g->ny, &ap) || !make_axis_plan(g->nz, &ap))
    fail(PT_INVALID_ARG, "grid dimensions must be 2..64 and 2,3,5-smooth");
  for (int a = 0; a < 3; ++a)
    if (!(g->L[a] > 0) || !std::isfinite(g->L[a])) fail(PT_INVALID_ARG, "cell lengths must be positive");
}

// integer frequency of index i on an n-point axis, wrapped to [-n/2, n/2)
static inline int wrapped(int i, int n) { return i < (n + 1) / 2 ? i : i - n; }

FftTables::~FftTables() {
  cudaFree(tw);
  cudaFree(g2);
  cudaFree(g2d);
}

template <class T>
static void fill_tables(FftTables* t, const pt_grid& g) {
  const int ns[3] = {g.nx, g.ny, g.nz};
  std::vector<cx<T>> tw;
  std::vector<T> g2;
  std::vector<double> g2d;
  for (int a = 0; a < 3; ++a) {
    const int n = ns[a];
    for (int i = 0; i < n; ++i) {
      const double ang = -2.0 * M_PI * double(i) / double(n);
      tw.push_back(cx<T>{T(std::cos(ang)), T(std::sin(ang))});
      const double ga = 2.0 * M_PI * wrapped(i, n) / g.L[a];
      g2.push_back(T(ga * ga));
      g2d.push_back(ga * ga);
    }
  }
  PT_CUDA_CHECK(cudaMalloc(&t->g2d, g2d.size() * sizeof(double)));
  PT_CUDA_CHECK(cudaMemcpy(t->g2d, g2d.data(), g2d.size() * sizeof(double), cudaMemcpyHostToDevice));
  PT_CUDA_CHECK(cudaMalloc(&t->tw, tw.size() * sizeof(cx<T>)));
  PT_CUDA_CHECK(cudaMalloc(&t->g2, g2.size() * sizeof(T)));
  PT_CUDA_CHECK(cudaMemcpy(t->tw, tw.data(), tw.size() * sizeof(cx<T>), cudaMemcpyHostToDevice));
  PT_CUDA_CHECK(cudaMemcpy(t->g2, g2.data(), g2.size() * sizeof(T), cudaMemcpyHostToDevice));
}

const FftTables& fft_tables(pt_ctx* ctx, const pt_grid& g, pt_precision prec) {
  const bool dbl = (prec == PT_FP64);
  char key[160];
  snprintf(key, sizeof(key), "fft:%d:%d:%d:%.17g:%.17g:%.17g:%d", g.nx, g.ny, g.nz, g.L[0], g.L[1], g.L[2],
           int(dbl));
  auto it = ctx->caches.find(key);
  if (it != ctx->caches.end()) return *std::static_pointer_cast<FftTables>(it->second);
  auto t = std::make_shared<FftTables>();
  t->grid = g;
  t->plan = make_grid_plan(g);
  t->prec = dbl ? PT_FP64 : PT_FP32;
  if (dbl) fill_tables<double>(t.get(), g);
  else fill_tables<float>(t.get(), g);
  ctx->caches[key] = t;
  return *t;
}

struct KernelTableImpl {
  void* d = nullptr;
  ~KernelTableImpl() { cudaFree(d); }
};

double kernel_value(const pt_kernel& k, double G2) {
  if (G2 == 0.0) {
    if (k.type == 0) return std::isfinite(k.g0) ? k.g0 : 0.0;
    return std::isfinite(k.g0) ? k.g0 : M_PI / (k.mu * k.mu);
  }
  const double base = 4.0 * M_PI / G2;
  if (k.type == 0) return base;
  return base * (-std::expm1(-G2 / (4.0 * k.mu * k.mu)));
}

const void* kernel_table(pt_ctx* ctx, const pt_grid& g, const pt_kernel& k, pt_precision prec) {
  const bool dbl = (prec == PT_FP64);
  char key[200];
  snprintf(key, sizeof(key), "ktab:%d:%d:%d:%.17g:%.17g:%.17g:%d:%.17g:%.17g:%d", g.nx, g.ny, g.nz, g.L[0],
           g.L[1], g.L[2], k.type, k.mu, k.g0, int(dbl));
  auto it = ctx->caches.find(key);
  if (it != ctx->caches.end()) return std::static_pointer_cast<KernelTableImpl>(it->second)->d;
  const size_t ng = ng_of(g);
  std::vector<double> kt(ng);
  for (int z = 0; z < g.nz; ++z) {
    const double gz = 2.0 * M_PI * wrapped(z, g.nz) / g.L[2];
    for (int y = 0; y < g.ny; ++y) {
      const double gy = 2.0 * M_PI * wrapped(y, g.ny) / g.L[1];
      for (int x = 0; x < g.nx; ++x) {
        const double gx = 2.0 * M_PI * wrapped(x, g.nx) / g.L[0];
        kt[(size_t(z) * g.ny + y) * g.nx + x] = kernel_value(k, gx * gx + gy * gy + gz * gz) / double(ng);
      }
    }
  }
  auto t = std::make_shared<KernelTableImpl>();
  if (dbl) {
    PT_CUDA_CHECK(cudaMalloc(&t->d, ng * sizeof(double)));
    PT_CUDA_CHECK(cudaMemcpy(t->d, kt.data(), ng * sizeof(double), cudaMemcpyHostToDevice));
  } else {
    std::vector<float> kf(kt.begin(), kt.end());
    PT_CUDA_CHECK(cudaMalloc(&t->d, ng * sizeof(float)));
    PT_CUDA_CHECK(cudaMemcpy(t->d, kf.data(), ng * sizeof(float), cudaMemcpyHostToDevice));
  }
  ctx->caches[key] = t;
  return t->d;
}

}  // namespace pt
